// field_tile.cuh -- one tile of the fused Faraday + Ampere update, shared by the
// per-step field kernel and the persistent ensemble kernel.
//
//   B^{n+1/2} = B^{n-1/2} - dt d_E x E^n          (Eq. (1), App. B Eq. (B.1))
//   E^{n+1}   = E^n + dt (d_B x B^{n+1/2} - J)     (Eq. (1), App. B Eq. (B.2))
//
// E^n and B^{n-1/2} of the tile plus the halo of the two wide x1 stencils
// (2M-1 cells each side in x1, one cell in x2/x3) are staged in shared memory;
// every value of E, B, J is read from HBM once and E, B are written once (15
// values per cell); halo re-reads hit L2.  Inputs and outputs are separate
// buffers, because neighbouring tiles read this tile's cells as their halo.
#pragma once
#include "common.cuh"

namespace pic {

// Periodic index for a region that may reach past the grid on either side (any
// number of periods: the loops run zero or one time except on tiny grids).
__device__ __forceinline__ int pwrap(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// CG = true reads through L2 only (ld.global.cg): a persistent kernel reads, in
// a later step, buffers other SMs wrote, and must not hit stale L1 lines.
template <bool CG, typename T>
__device__ __forceinline__ T gload(const T* p) {
  if (CG) return __ldcg(p);
  return *p;
}

struct FieldDims {
  int n1, n2, n3;
};

// Copy W consecutive (periodic) values of a grid row starting at column g0 into
// shared memory, one warp per row.  Rows that do not cross the periodic seam
// (all but the edge tiles) take the unrolled path with several loads in flight.
template <bool CG, typename T>
__device__ __forceinline__ void stage_row(T* dst, const T* src, int g0, int W, int n1, int lane) {
  if (g0 >= 0 && g0 + W <= n1) {
    const T* s = src + g0;
#pragma unroll 4
    for (int l1 = lane; l1 < W; l1 += 32) dst[l1] = gload<CG>(s + l1);
  } else {
    for (int l1 = lane; l1 < W; l1 += 32) dst[l1] = gload<CG>(src + pwrap(g0 + l1, n1));
  }
}

// Update tile number `tile` (x1 fastest over ceil(n/T) tiles per axis).
// j may be null (no current); with zero_j the tile's current is cleared after
// it is read (ready for the next step's deposit).  smem holds 3*(nE + nB) values.
template <typename T, int NDIM, bool CG>
__device__ __forceinline__ void field_tile(const T* const* e, const T* const* b, T* const* j,
                                           T* const* eo, T* const* bo, FieldDims dim,
                                           const StencilArgs<T>& s, T dt, int TX, int TY, int TZ,
                                           int tile, T* sm, bool zero_j = false) {
  const int M = s.M;
  const int n1 = dim.n1, n2 = dim.n2, n3 = (NDIM == 3) ? dim.n3 : 1;
  const int ntx = (n1 + TX - 1) / TX, nty = (n2 + TY - 1) / TY;
  int tb = tile;
  const int tx = tb % ntx;
  tb /= ntx;
  const int ty = tb % nty;
  const int tz = tb / nty;
  const int i0 = tx * TX, j0 = ty * TY, k0 = tz * TZ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

  // regions: E^n over [i0-2M+1, i0+TX+2M-1) x [j0-1, j0+TY+1) (x [k0-1, k0+TZ+1)),
  //          B over [i0-M, i0+TX+M-1) x [j0-1, j0+TY) (x [k0-1, k0+TZ))
  const int WE1 = TX + 4 * M - 2, WE2 = TY + 2, WE3 = (NDIM == 3) ? TZ + 2 : 1;
  const int WB1 = TX + 2 * M - 1, WB2 = TY + 1, WB3 = (NDIM == 3) ? TZ + 1 : 1;
  const int oE1 = i0 - 2 * M + 1, oB1 = i0 - M;
  const int nE = WE1 * WE2 * WE3, nB = WB1 * WB2 * WB3;
  T* sE = sm;            // [3][WE3][WE2][WE1]
  T* sB = sm + 3 * nE;   // [3][WB3][WB2][WB1]

  for (int row = warp; row < 3 * WE2 * WE3; row += nwarp) {
    const int l2 = row % WE2, r = row / WE2;
    const int l3 = r % WE3, c = r / WE3;
    const int gj = pwrap(j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(k0 - 1 + l3, n3) : 0;
    stage_row<CG>(sE + row * WE1, e[c] + ((int64_t)gk * n2 + gj) * n1, oE1, WE1, n1, lane);
  }
  for (int row = warp; row < 3 * WB2 * WB3; row += nwarp) {
    const int l2 = row % WB2, r = row / WB2;
    const int l3 = r % WB3, c = r / WB3;
    const int gj = pwrap(j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(k0 - 1 + l3, n3) : 0;
    stage_row<CG>(sB + row * WB1, b[c] + ((int64_t)gk * n2 + gj) * n1, oB1, WB1, n1, lane);
  }
  __syncthreads();

  // Faraday over the B region: B^{n+1/2} = B - dt d_E x E (coefficients pre-scaled)
  const int sE2 = WE1, sE3 = WE1 * WE2;
  const T* E1 = sE;
  const T* E2 = sE + nE;
  const T* E3 = sE + 2 * nE;
  for (int row = warp; row < WB2 * WB3; row += nwarp) {
    const int l2 = row % WB2, l3 = row / WB2;
    for (int l1 = lane; l1 < WB1; l1 += 32) {
      const int q = row * WB1 + l1;
      const int ei = l3 * sE3 + l2 * sE2 + (l1 + M - 1);  // this B point in the E region
      T dE3 = 0, dE2 = 0;
#pragma unroll 8
      for (int m = 1; m <= M; ++m) {
        const T c = s.kE[m - 1];
        dE3 += c * (E3[ei + m] - E3[ei - m + 1]);
        dE2 += c * (E2[ei + m] - E2[ei - m + 1]);
      }
      const T d2E3 = s.y2 * (E3[ei + sE2] - E3[ei]);
      const T d2E1 = s.y2 * (E1[ei + sE2] - E1[ei]);
      T d3E2 = 0, d3E1 = 0;
      if (NDIM == 3) {
        d3E2 = s.y3 * (E2[ei + sE3] - E2[ei]);
        d3E1 = s.y3 * (E1[ei + sE3] - E1[ei]);
      }
      sB[q] -= d2E3 - d3E2;            // B1 -= dt (d2 E3 - d3 E2)
      sB[nB + q] -= d3E1 - dE3;        // B2 -= dt (d3 E1 - d^E1 E3)
      sB[2 * nB + q] -= dE2 - d2E1;    // B3 -= dt (d^E1 E2 - d2 E1)
    }
  }
  __syncthreads();

  // Ampere over the tile: E^{n+1} = E + dt (d_B x B^{n+1/2} - J); write E and B
  const int sB2 = WB1, sB3 = WB1 * WB2;
  const T* B1 = sB;
  const T* B2 = sB + nB;
  const T* B3 = sB + 2 * nB;
  const int TZe = (NDIM == 3) ? TZ : 1;
  for (int row = warp; row < TY * TZe; row += nwarp) {
    const int o2 = row % TY, o3 = row / TY;
    const int gj = j0 + o2, gk = k0 + o3;
    if (gj >= n2 || (NDIM == 3 && gk >= n3)) continue;
    const int64_t rowoff = ((int64_t)gk * n2 + gj) * n1;
    for (int o1 = lane; o1 < TX; o1 += 32) {
      const int gi = i0 + o1;
      if (gi >= n1) break;
      const int bi = (NDIM == 3 ? (o3 + 1) * sB3 : 0) + (o2 + 1) * sB2 + (o1 + M);
      const int ei = (NDIM == 3 ? (o3 + 1) * sE3 : 0) + (o2 + 1) * sE2 + (o1 + 2 * M - 1);
      T dB3 = 0, dB2 = 0;
#pragma unroll 8
      for (int m = 1; m <= M; ++m) {
        const T c = s.kB[m - 1];
        dB3 += c * (B3[bi + m - 1] - B3[bi - m]);
        dB2 += c * (B2[bi + m - 1] - B2[bi - m]);
      }
      const T d2B3 = s.y2 * (B3[bi] - B3[bi - sB2]);
      const T d2B1 = s.y2 * (B1[bi] - B1[bi - sB2]);
      T d3B2 = 0, d3B1 = 0;
      if (NDIM == 3) {
        d3B2 = s.y3 * (B2[bi] - B2[bi - sB3]);
        d3B1 = s.y3 * (B1[bi] - B1[bi - sB3]);
      }
      const int64_t gidx = rowoff + gi;
      const T j1 = j ? gload<CG>(j[0] + gidx) : (T)0;
      const T j2 = j ? gload<CG>(j[1] + gidx) : (T)0;
      const T j3 = j ? gload<CG>(j[2] + gidx) : (T)0;
      if (j && zero_j) {
        j[0][gidx] = (T)0;
        j[1][gidx] = (T)0;
        j[2][gidx] = (T)0;
      }
      eo[0][gidx] = E1[ei] + ((d2B3 - d3B2) - dt * j1);
      eo[1][gidx] = E2[ei] + ((d3B1 - dB3) - dt * j2);
      eo[2][gidx] = E3[ei] + ((dB2 - d2B1) - dt * j3);
      bo[0][gidx] = B1[bi];
      bo[1][gidx] = B2[bi];
      bo[2][gidx] = B3[bi];
    }
  }
}

// shared-memory values a tile needs
__host__ __device__ inline size_t field_tile_smem_elems(int ndim, int TX, int TY, int TZ, int M) {
  const size_t nE = (size_t)(TX + 4 * M - 2) * (TY + 2) * (ndim == 3 ? TZ + 2 : 1);
  const size_t nB = (size_t)(TX + 2 * M - 1) * (TY + 1) * (ndim == 3 ? TZ + 1 : 1);
  return 3 * (nE + nB);
}

}  // namespace pic
