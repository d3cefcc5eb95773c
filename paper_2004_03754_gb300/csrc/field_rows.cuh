// field_rows.cuh -- one row of the 2D field update streamed along x2 by a warp,
// shared by the per-step field kernel and the persistent ensemble kernel.
//
//   B^{n+1/2} = B^{n-1/2} - dt d_E x E^n          (Eq. (1), App. B Eq. (B.1))
//   E^{n+1}   = E^n + dt (d_B x B^{n+1/2} - J)     (Eq. (1), App. B Eq. (B.2))
#pragma once
#include "common.cuh"
#include "field_tile.cuh"
#include "march_layout.cuh"

namespace pic {

// Rows of a strip streamed along x2 (march_row in one warp, or march_faraday and
// march_ampere in two).  Faraday forms B^{n+1/2} row t from E rows t (stage sq)
// and t+1 (stage sq1) and B^{n-1/2} row t; then, for q >= 1, Ampere forms
// E^{n+1} row t from B^{n+1/2} rows t and t-1 and stores it with B^{n+1/2} row t into the
// strip's columns [i0, min(i0+SW, n1)) of eo/bo (rows of ld >= n1 values; 16-byte
// vector stores for whole groups when ld is a multiple of 16 bytes, scalar
// stores otherwise; nothing is stored past column n1 - 1).
// Stage layout: E1 E2 E3 rows (WE values from column i0-DB-DE), B1 B2 B3 rows
// (WB values from column i0-DB), J1 J2 J3 rows (SW values from column i0; the
// ensemble kernel stages J, the per-step kernel reads it into registers and
// takes march_faraday with march_ampere_jr on stages without J rows).
// has_j = false: no current (J taken as zero); jclear (nullable): the current
// arrays, whose row t is cleared once read.  gh > 0: the rows of eo/bo carry gh
// ghost columns on each side (column c of the periodic row also at c - n1 for
// c >= n1 - gh and at c + n1 for c < gh), which are written with the row.

// Faraday part of a row: B^{n+1/2} row t over the strip's B region into bn
// ([3][WB]) from E rows t (stage sq) and t+1 (stage sq1) and B^{n-1/2} row t.
template <typename T, int MT>
__device__ __forceinline__ void march_faraday(const T* sq, const T* sq1, T* bn, int WE, int WB,
                                              const StencilArgs<T>& s, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  for (int gq = lane; gq < WB / V; gq += 32) {
    const int col = gq * V, ec = col + RC.DE;
    T dE3[V], dE2[V];
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE3, sq + 2 * WE + col, s.kE);
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE2, sq + WE + col, s.kE);
    T a[V], b_[V], c_[V], d_[V], b1[V], b2[V], b3[V];
    vld(a, sq1 + 2 * WE + ec);
    vld(b_, sq + 2 * WE + ec);
    vld(c_, sq1 + ec);
    vld(d_, sq + ec);
    const T* bo_ = sq + 3 * WE + col;
    vld(b1, bo_);
    vld(b2, bo_ + WB);
    vld(b3, bo_ + 2 * WB);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T d2E3 = s.y2 * (a[v] - b_[v]);
      const T d2E1 = s.y2 * (c_[v] - d_[v]);
      const T d3E2 = 0, d3E1 = 0;
      b1[v] -= d2E3 - d3E2;
      b2[v] -= d3E1 - dE3[v];
      b3[v] -= dE2[v] - d2E1;
    }
    vst(bn + col, b1);
    vst(bn + WB + col, b2);
    vst(bn + 2 * WB + col, b3);
  }
}

// Ampere part of a row: E^{n+1} row t from B^{n+1/2} rows t (bn) and t-1 (bm),
// E^n and J row t of stage sq; stores E^{n+1} and B^{n+1/2} row t (see march_row).
template <typename T, int MT>
__device__ __forceinline__ void march_ampere(const T* sq, const T* bn, const T* bm, int t, int i0,
                                             int n1, int ld, int gh, int WE, int WB, int SW,
                                             const StencilArgs<T>& s, T dt, T* const* eo,
                                             T* const* bo, bool has_j, T* const* jclear, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  const T* sj = sq + 3 * WE + 3 * WB;
  const int nA = min(SW, n1 - i0);  // columns of the strip inside the grid
  const int ngA = (nA + V - 1) / V;
  const bool vec = (ld % V) == 0;   // rows start on 16-byte boundaries
  for (int gq = lane; gq < ngA; gq += 32) {
    const int oc = gq * V;
    const int bc = oc + RC.DB, ec = oc + RC.DB + RC.DE;
    T dB3[V], dB2[V];
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB3, bn + 2 * WB + oc, s.kB);
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB2, bn + WB + oc, s.kB);
    T b1[V], b2[V], b3[V], b1m[V], b3m[V], j1[V], j2[V], j3[V], e1[V], e2[V], e3[V];
    vld(b1, bn + bc);
    vld(b2, bn + WB + bc);
    vld(b3, bn + 2 * WB + bc);
    vld(b1m, bm + bc);
    vld(b3m, bm + 2 * WB + bc);
    if (has_j) {
      vld(j1, sj + oc);
      vld(j2, sj + SW + oc);
      vld(j3, sj + 2 * SW + oc);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) j1[v] = j2[v] = j3[v] = (T)0;
    }
    vld(e1, sq + ec);
    vld(e2, sq + WE + ec);
    vld(e3, sq + 2 * WE + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T d2B3 = s.y2 * (b3[v] - b3m[v]);
      const T d2B1 = s.y2 * (b1[v] - b1m[v]);
      const T d3B2 = 0, d3B1 = 0;
      e1[v] = e1[v] + ((d2B3 - d3B2) - dt * j1[v]);
      e2[v] = e2[v] + ((d3B1 - dB3[v]) - dt * j2[v]);
      e3[v] = e3[v] + ((dB2[v] - d2B1) - dt * j3[v]);
    }
    const int64_t gidx = (int64_t)t * ld + i0 + oc;
    if (vec && oc + V <= nA) {  // a whole group inside the run (columns past n1 may be ghosts)
      vst(eo[0] + gidx, e1);
      vst(eo[1] + gidx, e2);
      vst(eo[2] + gidx, e3);
      vst(bo[0] + gidx, b1);
      vst(bo[1] + gidx, b2);
      vst(bo[2] + gidx, b3);
      if (jclear) {
        const T z[V] = {};
        vst(jclear[0] + gidx, z);
        vst(jclear[1] + gidx, z);
        vst(jclear[2] + gidx, z);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (oc + v >= nA) break;
        eo[0][gidx + v] = e1[v];
        eo[1][gidx + v] = e2[v];
        eo[2][gidx + v] = e3[v];
        bo[0][gidx + v] = b1[v];
        bo[1][gidx + v] = b2[v];
        bo[2][gidx + v] = b3[v];
        if (jclear) {
          jclear[0][gidx + v] = (T)0;
          jclear[1][gidx + v] = (T)0;
          jclear[2][gidx + v] = (T)0;
        }
      }
    }
    if (gh > 0 && (i0 + oc < gh || i0 + oc + V > n1 - gh)) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int gi = i0 + oc + v;
        if (gi >= n1) break;
        const int64_t k = gidx + v;
        if (gi < gh) {
          eo[0][k + n1] = e1[v];
          eo[1][k + n1] = e2[v];
          eo[2][k + n1] = e3[v];
          bo[0][k + n1] = b1[v];
          bo[1][k + n1] = b2[v];
          bo[2][k + n1] = b3[v];
        }
        if (gi >= n1 - gh) {
          eo[0][k - n1] = e1[v];
          eo[1][k - n1] = e2[v];
          eo[2][k - n1] = e3[v];
          bo[0][k - n1] = b1[v];
          bo[1][k - n1] = b2[v];
          bo[2][k - n1] = b3[v];
        }
      }
    }
  }
}

// Ampere part of a row for the per-step 2D kernel (rows of pitch n1, no ghost
// columns): as march_ampere, with J row t read from global memory rather than
// staged -- the lane's first NGJ column groups already in jr (loaded before the
// row's Faraday so that it covers the latency), later groups from jg (the three
// components' rows at column i0).
template <typename T, int MT, int NGJ>
__device__ __forceinline__ void march_ampere_jr(const T* sq, const T* bn, const T* bm, int t,
                                                int i0, int n1, int WE, int WB, int SW,
                                                const StencilArgs<T>& s, T dt, T* const* eo,
                                                T* const* bo, const T (*jr)[3][VecOf<T>::V],
                                                const T* const* jg, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  const int nA = min(SW, n1 - i0);  // columns of the strip inside the grid
  const int ngA = (nA + V - 1) / V;
  const bool vec = (n1 % V) == 0;
  auto group = [&](int gq, const T* j1, const T* j2, const T* j3) {
    const int oc = gq * V;
    const int bc = oc + RC.DB, ec = oc + RC.DB + RC.DE;
    T dB3[V], dB2[V];
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB3, bn + 2 * WB + oc, s.kB);
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB2, bn + WB + oc, s.kB);
    T b1[V], b2[V], b3[V], b1m[V], b3m[V], e1[V], e2[V], e3[V];
    vld(b1, bn + bc);
    vld(b2, bn + WB + bc);
    vld(b3, bn + 2 * WB + bc);
    vld(b1m, bm + bc);
    vld(b3m, bm + 2 * WB + bc);
    vld(e1, sq + ec);
    vld(e2, sq + WE + ec);
    vld(e3, sq + 2 * WE + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T d2B3 = s.y2 * (b3[v] - b3m[v]);
      const T d2B1 = s.y2 * (b1[v] - b1m[v]);
      const T d3B2 = 0, d3B1 = 0;
      e1[v] = e1[v] + ((d2B3 - d3B2) - dt * j1[v]);
      e2[v] = e2[v] + ((d3B1 - dB3[v]) - dt * j2[v]);
      e3[v] = e3[v] + ((dB2[v] - d2B1) - dt * j3[v]);
    }
    const int64_t gidx = (int64_t)t * n1 + i0 + oc;
    if (vec && oc + V <= nA) {
      vst(eo[0] + gidx, e1);
      vst(eo[1] + gidx, e2);
      vst(eo[2] + gidx, e3);
      vst(bo[0] + gidx, b1);
      vst(bo[1] + gidx, b2);
      vst(bo[2] + gidx, b3);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (oc + v >= nA) break;
        eo[0][gidx + v] = e1[v];
        eo[1][gidx + v] = e2[v];
        eo[2][gidx + v] = e3[v];
        bo[0][gidx + v] = b1[v];
        bo[1][gidx + v] = b2[v];
        bo[2][gidx + v] = b3[v];
      }
    }
  };
#pragma unroll
  for (int m = 0; m < NGJ; ++m) {
    const int gq = lane + 32 * m;
    if (gq < ngA) group(gq, jr[m][0], jr[m][1], jr[m][2]);
  }
  for (int gq = lane + 32 * NGJ; gq < ngA; gq += 32) {
    T j1[V], j2[V], j3[V];
    vld_global<true>(j1, jg[0] + gq * V);
    vld_global<true>(j2, jg[1] + gq * V);
    vld_global<true>(j3, jg[2] + gq * V);
    group(gq, j1, j2, j3);
  }
}

// One row of a strip streamed along x2 by one warp: Faraday into the two-row
// ring slot q&1 of bnew, then (q >= 1) Ampere for row t (march_faraday,
// march_ampere).
template <typename T, int MT>
__device__ __forceinline__ void march_row(const T* sq, const T* sq1, T* bnew, int q, int t, int i0,
                                          int n1, int ld, int gh, int WE, int WB, int SW,
                                          const StencilArgs<T>& s, T dt, T* const* eo,
                                          T* const* bo, bool has_j, T* const* jclear, int lane) {
  T* bn = bnew + (q & 1) * 3 * WB;
  march_faraday<T, MT>(sq, sq1, bn, WE, WB, s, lane);
  __syncwarp();
  if (q < 1) return;
  march_ampere<T, MT>(sq, bn, bnew + ((q - 1) & 1) * 3 * WB, t, i0, n1, ld, gh, WE, WB, SW, s, dt,
                      eo, bo, has_j, jclear, lane);
}

}  // namespace pic

namespace pic {

// One x2 row of a 3D strip streamed along x2 by one warp, for the x3 plane k of
// the item.  Stage layout (row t): E1 E2 E3 rows at planes k-1, k, k+1
// (index 3p + c, p = 0, 1, 2; WE values from column i0-DB-DE), B1 B2 B3 rows
// at planes k-1, k (index 3p + c, WB values from column i0-DB), J1 J2 J3 rows
// at plane k (SW values from column i0).  Faraday forms B^{n+1/2} row t of plane
// k into the two-row ring bnew (slot q&1) and, of plane k-1, the B1 and B2 that
// Ampere's x3 differences need into bk; then, for q >= 1, Ampere forms E^{n+1}
// row t of plane k and stores it with B^{n+1/2} into eo / bo (rows of pitch
// n1, plane stride n1 n2).  The operations and their order per value are the
// field tile's (tile_compute), so the results are bit-identical to it.
template <typename T, int MT>
__device__ __forceinline__ void march_row3(const T* sq, const T* sq1, T* bnew, T* bk, int q,
                                           int t, int k, int i0, int n1, int n2, int WE, int WB,
                                           int SW, const StencilArgs<T>& s, T dt, T* const* eo,
                                           T* const* bo, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  auto Er = [&](const T* st, int p, int c) { return st + (3 * p + c) * WE; };
  auto Br = [&](const T* st, int p, int c) { return st + 9 * WE + (3 * p + c) * WB; };
  T* bn = bnew + (q & 1) * 3 * WB;
  for (int gq = lane; gq < WB / V; gq += 32) {
    const int col = gq * V, ec = col + RC.DE;
    // plane k
    T dE3[V], dE2[V];
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE3, Er(sq, 1, 2) + col, s.kE);
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE2, Er(sq, 1, 1) + col, s.kE);
    T a[V], b_[V], c_[V], d_[V], b1[V], b2[V], b3[V];
    T d2E3[V], d2E1[V], d3E2[V], d3E1[V];
    vld(a, Er(sq1, 1, 2) + ec);
    vld(b_, Er(sq, 1, 2) + ec);
    vld(c_, Er(sq1, 1, 0) + ec);
    vld(d_, Er(sq, 1, 0) + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d2E3[v] = s.y2 * (a[v] - b_[v]);
      d2E1[v] = s.y2 * (c_[v] - d_[v]);
    }
    vld(a, Er(sq, 2, 1) + ec);
    vld(b_, Er(sq, 1, 1) + ec);
    vld(c_, Er(sq, 2, 0) + ec);
    vld(d_, Er(sq, 1, 0) + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d3E2[v] = s.y3 * (a[v] - b_[v]);
      d3E1[v] = s.y3 * (c_[v] - d_[v]);
    }
    vld(b1, Br(sq, 1, 0) + col);
    vld(b2, Br(sq, 1, 1) + col);
    vld(b3, Br(sq, 1, 2) + col);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      b1[v] -= d2E3[v] - d3E2[v];
      b2[v] -= d3E1[v] - dE3[v];
      b3[v] -= dE2[v] - d2E1[v];
    }
    vst(bn + col, b1);
    vst(bn + WB + col, b2);
    vst(bn + 2 * WB + col, b3);
  }
  // plane k-1: B1 and B2 only, at the strip's own columns (the x3 differences of
  // Ampere read nothing else), one pass of the warp for SW = 128 FP32 columns
  for (int gq = lane; gq < SW / V; gq += 32) {
    const int col = RC.DB + gq * V, ec = col + RC.DE;
    T dE3[V], a[V], b_[V], c_[V], d_[V], b1[V], b2[V], d2E3[V], d3E2[V], d3E1[V];
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE3, Er(sq, 0, 2) + col, s.kE);
    vld(a, Er(sq1, 0, 2) + ec);
    vld(b_, Er(sq, 0, 2) + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) d2E3[v] = s.y2 * (a[v] - b_[v]);
    vld(a, Er(sq, 1, 1) + ec);
    vld(b_, Er(sq, 0, 1) + ec);
    vld(c_, Er(sq, 1, 0) + ec);
    vld(d_, Er(sq, 0, 0) + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d3E2[v] = s.y3 * (a[v] - b_[v]);
      d3E1[v] = s.y3 * (c_[v] - d_[v]);
    }
    vld(b1, Br(sq, 0, 0) + col);
    vld(b2, Br(sq, 0, 1) + col);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      b1[v] -= d2E3[v] - d3E2[v];
      b2[v] -= d3E1[v] - dE3[v];
    }
    vst(bk + col, b1);
    vst(bk + WB + col, b2);
  }
  __syncwarp();
  if (q < 1) return;
  const T* bm = bnew + ((q - 1) & 1) * 3 * WB;  // B^{n+1/2} row t-1, plane k
  const T* sj = sq + 9 * WE + 6 * WB;
  const int nA = min(SW, n1 - i0);
  const int ngA = (nA + V - 1) / V;
  const int64_t rowbase = ((int64_t)k * n2 + t) * n1 + i0;
  for (int gq = lane; gq < ngA; gq += 32) {
    const int oc = gq * V;
    const int bc = oc + RC.DB, ec = oc + RC.DB + RC.DE;
    T dB3[V], dB2[V];
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB3, bn + 2 * WB + oc, s.kB);
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB2, bn + WB + oc, s.kB);
    T b1[V], b2[V], b3[V], b1m[V], b3m[V], b1k[V], b2k[V], j1[V], j2[V], j3[V], e1[V], e2[V], e3[V];
    vld(b1, bn + bc);
    vld(b2, bn + WB + bc);
    vld(b3, bn + 2 * WB + bc);
    vld(b1m, bm + bc);
    vld(b3m, bm + 2 * WB + bc);
    vld(b1k, bk + bc);
    vld(b2k, bk + WB + bc);
    vld(j1, sj + oc);
    vld(j2, sj + SW + oc);
    vld(j3, sj + 2 * SW + oc);
    vld(e1, Er(sq, 1, 0) + ec);
    vld(e2, Er(sq, 1, 1) + ec);
    vld(e3, Er(sq, 1, 2) + ec);
    T d2B3[V], d2B1[V], d3B2[V], d3B1[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d2B3[v] = s.y2 * (b3[v] - b3m[v]);
      d2B1[v] = s.y2 * (b1[v] - b1m[v]);
      d3B2[v] = s.y3 * (b2[v] - b2k[v]);
      d3B1[v] = s.y3 * (b1[v] - b1k[v]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      e1[v] = e1[v] + ((d2B3[v] - d3B2[v]) - dt * j1[v]);
      e2[v] = e2[v] + ((d3B1[v] - dB3[v]) - dt * j2[v]);
      e3[v] = e3[v] + ((dB2[v] - d2B1[v]) - dt * j3[v]);
    }
    const int64_t gidx = rowbase + oc;
    if (oc + V <= nA) {
      vst(eo[0] + gidx, e1);
      vst(eo[1] + gidx, e2);
      vst(eo[2] + gidx, e3);
      vst(bo[0] + gidx, b1);
      vst(bo[1] + gidx, b2);
      vst(bo[2] + gidx, b3);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (oc + v >= nA) break;
        eo[0][gidx + v] = e1[v];
        eo[1][gidx + v] = e2[v];
        eo[2][gidx + v] = e3[v];
        bo[0][gidx + v] = b1[v];
        bo[1][gidx + v] = b2[v];
        bo[2][gidx + v] = b3[v];
      }
    }
  }
}

}  // namespace pic

namespace pic {

// Plane-group rows (field_planes3_kernel): the layout is Planes3 (march_layout.cuh).

// Faraday part of row t for warp w of a group of Pg planes: B^{n+1/2} of plane
// k0+w over the B region into bn ([3][WB]) and, for the warp's share of the
// strip's columns, B1 and B2 of plane k0-1 into brec ([2][WB], B region
// columns DB .. DB+SW).  E rows t from stage sq, E rows t+1 from sq1.  Every
// task of a warp runs the same instructions (the plane-k0-1 tasks also form a
// B3 that is not stored), and each value takes the field tile's operations in
// its order (tile_compute), so the results are bit-identical to it.
template <typename T, int MT>
__device__ __forceinline__ void planes3_faraday(const T* sq, const T* sq1, T* bn, T* brec, int w,
                                                int Pg, const Planes3& L, const StencilArgs<T>& s,
                                                int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  const int WB = L.WB;
  const int nOwn = WB / V, nRec = L.SW / V;
  const int per = (nRec + Pg - 1) / Pg, rs = w * per;
  const int cnt = max(0, min(per, nRec - rs));
  for (int task = lane; task < nOwn + cnt; task += 32) {
    const bool own = task < nOwn;
    const int pe = own ? w + 1 : 0;
    const int col = own ? task * V : RC.DB + (rs + task - nOwn) * V;
    const int ec = col + RC.DE;
    const T* E1 = sq + L.er(pe, 0);
    const T* E2 = sq + L.er(pe, 1);
    const T* E3 = sq + L.er(pe, 2);
    T dE3[V], dE2[V];
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE3, E3 + col, s.kE);
    x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE2, E2 + col, s.kE);
    T a[V], b_[V], c_[V], d_[V], b1[V], b2[V], b3[V];
    T d2E3[V], d2E1[V], d3E2[V], d3E1[V];
    vld(a, sq1 + L.er(pe, 2) + ec);
    vld(b_, E3 + ec);
    vld(c_, sq1 + L.er(pe, 0) + ec);
    vld(d_, E1 + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d2E3[v] = s.y2 * (a[v] - b_[v]);
      d2E1[v] = s.y2 * (c_[v] - d_[v]);
    }
    vld(a, sq + L.er(pe + 1, 1) + ec);
    vld(b_, E2 + ec);
    vld(c_, sq + L.er(pe + 1, 0) + ec);
    vld(d_, E1 + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d3E2[v] = s.y3 * (a[v] - b_[v]);
      d3E1[v] = s.y3 * (c_[v] - d_[v]);
    }
    // B1, B2, B3 of plane pe (for pe = 0 the third row read is another plane's
    // B1: its B3 is not stored)
    const T* Bq = sq + L.br(pe, 0);
    vld(b1, Bq + col);
    vld(b2, Bq + WB + col);
    vld(b3, Bq + 2 * WB + col);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      b1[v] -= d2E3[v] - d3E2[v];
      b2[v] -= d3E1[v] - dE3[v];
      b3[v] -= dE2[v] - d2E1[v];
    }
    T* dst = own ? bn : brec;
    vst(dst + col, b1);
    vst(dst + WB + col, b2);
    if (own) vst(dst + 2 * WB + col, b3);
  }
}

// Ampere part of row t for warp w (plane k = k0+w): E^{n+1} from B^{n+1/2} row t
// of plane k (bn, [3][WB]), B1 B3 row t-1 of plane k over the strip (bm, [2][SW],
// overwritten here with those of row t), B1 B2 row t of plane k-1 (bk, component
// c at c WB), E^n of stage sq and J row t (jt: the three components' rows in
// global memory at column i0; the lane's first column group already in j0);
// stores E^{n+1} and B^{n+1/2} row t of plane k into eo / bo (rows of pitch n1,
// plane stride n1 n2) over the strip's columns [i0, min(i0+SW, n1)).
template <typename T, int MT>
__device__ __forceinline__ void planes3_ampere(const T* sq, const T* bn, T* bm, const T* bk,
                                               const T* const* jt, const T (*j0)[VecOf<T>::V],
                                               int w, int t, int k, int i0, int n1, int n2,
                                               const Planes3& L, const StencilArgs<T>& s, T dt,
                                               T* const* eo, T* const* bo, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  const int WB = L.WB, SW = L.SW;
  const int nA = min(SW, n1 - i0);
  const int ngA = (nA + V - 1) / V;
  const T* E1 = sq + L.er(w + 1, 0);
  const T* E2 = sq + L.er(w + 1, 1);
  const T* E3 = sq + L.er(w + 1, 2);
  const int64_t rowbase = ((int64_t)k * n2 + t) * n1 + i0;
  for (int gq = lane; gq < ngA; gq += 32) {
    const int oc = gq * V;
    const int bc = oc + RC.DB, ec = oc + RC.DB + RC.DE;
    T dB3[V], dB2[V];
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB3, bn + 2 * WB + oc, s.kB);
    x1_stencil<T, V, MT, RC.DB, RC.LB, 0>(dB2, bn + WB + oc, s.kB);
    T b1[V], b2[V], b3[V], b1m[V], b3m[V], b1k[V], b2k[V], j1[V], j2[V], j3[V], e1[V], e2[V], e3[V];
    vld(b1, bn + bc);
    vld(b2, bn + WB + bc);
    vld(b3, bn + 2 * WB + bc);
    vld(b1m, bm + oc);
    vld(b3m, bm + SW + oc);
    vld(b1k, bk + bc);
    vld(b2k, bk + WB + bc);
    if (gq < 32) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        j1[v] = j0[0][v];
        j2[v] = j0[1][v];
        j3[v] = j0[2][v];
      }
    } else {
      vld_global<true>(j1, jt[0] + oc);
      vld_global<true>(j2, jt[1] + oc);
      vld_global<true>(j3, jt[2] + oc);
    }
    vld(e1, E1 + ec);
    vld(e2, E2 + ec);
    vld(e3, E3 + ec);
    T d2B3[V], d2B1[V], d3B2[V], d3B1[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d2B3[v] = s.y2 * (b3[v] - b3m[v]);
      d2B1[v] = s.y2 * (b1[v] - b1m[v]);
      d3B2[v] = s.y3 * (b2[v] - b2k[v]);
      d3B1[v] = s.y3 * (b1[v] - b1k[v]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      e1[v] = e1[v] + ((d2B3[v] - d3B2[v]) - dt * j1[v]);
      e2[v] = e2[v] + ((d3B1[v] - dB3[v]) - dt * j2[v]);
      e3[v] = e3[v] + ((dB2[v] - d2B1[v]) - dt * j3[v]);
    }
    vst(bm + oc, b1);  // row t's B1, B3 for the next row's x2 differences
    vst(bm + SW + oc, b3);
    const int64_t gidx = rowbase + oc;
    if (oc + V <= nA) {
      vst(eo[0] + gidx, e1);
      vst(eo[1] + gidx, e2);
      vst(eo[2] + gidx, e3);
      vst(bo[0] + gidx, b1);
      vst(bo[1] + gidx, b2);
      vst(bo[2] + gidx, b3);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (oc + v >= nA) break;
        eo[0][gidx + v] = e1[v];
        eo[1][gidx + v] = e2[v];
        eo[2][gidx + v] = e3[v];
        bo[0][gidx + v] = b1[v];
        bo[1][gidx + v] = b2[v];
        bo[2][gidx + v] = b3[v];
      }
    }
  }
}

}  // namespace pic
