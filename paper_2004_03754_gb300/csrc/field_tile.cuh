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
#include "dfloat.cuh"

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
__host__ __device__ __forceinline__ T gload(const T* p) {
#ifdef __CUDA_ARCH__
  if constexpr (is_dfl<T>::value) {
    if (CG) {
      const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
      return T(q.x, q.y);
    }
  } else {
    if (CG) return __ldcg(p);
  }
#endif
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

// Register-blocked x1 stencils.  Each thread computes V = 16/sizeof(T)
// consecutive x1 outputs from a window of the row held in registers, loaded
// with 16-byte vector loads; the stencil is unrolled to MT >= M taps (the
// coefficients past M are zero).  Column ranges are multiples of V, so every
// vector access in shared memory is aligned.
template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
  static constexpr int V = 4;
};
template <>
struct VecOf<double> {
  static constexpr int V = 2;
};
template <>
struct VecOf<dfl> {
  static constexpr int V = 2;
};

__host__ __device__ constexpr int stencil_mt(int M) { return M <= 8 ? 8 : (M <= 16 ? 16 : 32); }
__host__ __device__ constexpr int ceil_to(int x, int v) { return (x + v - 1) / v * v; }

// Column reach of one tile along x1 for MT taps and V values per vector:
//   Ampere group g (V outputs) reads B over [g - DB, g - DB + LB),
//   Faraday group g reads E over [g - DE, g - DE + LE);
// the B region spans [i0 - DB, i0 - DB + WB), the E region [i0 - DB - DE, ... + WE).
struct Reach {
  int DE, LE, DB, LB;
  __host__ __device__ constexpr Reach(int MT, int V)
      : DE(ceil_to(MT - 1, V)), LE(ceil_to(ceil_to(MT - 1, V) + V + MT, V)), DB(ceil_to(MT, V)),
        LB(ceil_to(ceil_to(MT, V) + V + MT - 1, V)) {}
  __host__ __device__ constexpr int WB(int TX, int V) const { return TX - V + LB; }
  __host__ __device__ constexpr int WE(int TX, int V) const { return TX - V + LB - V + LE; }
};

// Geometry of one tile: E^n over columns [Es, Es+WE) x rows [j0-1, j0+TY+1)
// (x [k0-1, k0+TZ+1)), B over [Bs, Bs+WB) x [j0-1, j0+TY) (x [k0-1, k0+TZ)).
// Row r of a region sits at r * width in shared memory.
struct TileGeom {
  int i0, j0, k0;
  int Es, Bs;
  int WE, WE2, WE3, WB, WB2, WB3;
  int nE, nB;  // values per component in shared memory
};

template <typename T, int NDIM, int MT>
__device__ __forceinline__ TileGeom tile_geom(FieldDims dim, int TX, int TY, int TZ, int tile) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach R(MT, V);
  TileGeom G;
  const int ntx = (dim.n1 + TX - 1) / TX, nty = (dim.n2 + TY - 1) / TY;
  int tb = tile;
  const int tx = tb % ntx;
  tb /= ntx;
  const int ty = tb % nty;
  const int tz = tb / nty;
  G.i0 = tx * TX;
  G.j0 = ty * TY;
  G.k0 = tz * TZ;
  G.Bs = G.i0 - R.DB;
  G.Es = G.Bs - R.DE;
  G.WB = R.WB(TX, V);
  G.WE = R.WE(TX, V);
  G.WE2 = TY + 2;
  G.WE3 = (NDIM == 3) ? TZ + 2 : 1;
  G.WB2 = TY + 1;
  G.WB3 = (NDIM == 3) ? TZ + 1 : 1;
  G.nE = G.WE * G.WE2 * G.WE3;
  G.nB = G.WB * G.WB2 * G.WB3;
  return G;
}

// all threads: copy the two regions into shared memory (periodic wrap allowed)
template <bool CG, typename T, int NDIM>
__device__ __forceinline__ void tile_stage_sync(const T* const* e, const T* const* b, FieldDims dim,
                                                const TileGeom& G, T* sm) {
  const int n1 = dim.n1, n2 = dim.n2, n3 = (NDIM == 3) ? dim.n3 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  T* sE = sm;
  T* sB = sm + 3 * G.nE;
  for (int row = warp; row < 3 * G.WE2 * G.WE3; row += nwarp) {
    const int l2 = row % G.WE2, r = row / G.WE2;
    const int l3 = r % G.WE3, c = r / G.WE3;
    const int gj = pwrap(G.j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(G.k0 - 1 + l3, n3) : 0;
    stage_row<CG>(sE + row * G.WE, e[c] + ((int64_t)gk * n2 + gj) * n1, G.Es, G.WE, n1, lane);
  }
  for (int row = warp; row < 3 * G.WB2 * G.WB3; row += nwarp) {
    const int l2 = row % G.WB2, r = row / G.WB2;
    const int l3 = r % G.WB3, c = r / G.WB3;
    const int gj = pwrap(G.j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(G.k0 - 1 + l3, n3) : 0;
    stage_row<CG>(sB + row * G.WB, b[c] + ((int64_t)gk * n2 + gj) * n1, G.Bs, G.WB, n1, lane);
  }
}

// V consecutive values, 16-byte aligned
template <typename T>
__host__ __device__ __forceinline__ void vld(T* r, const T* p) {
  if constexpr (is_dfl<T>::value) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r[0] = T(q.x, q.y); r[1] = T(q.z, q.w);
  } else if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
  } else {
    const double2 q = *reinterpret_cast<const double2*>(p);
    r[0] = q.x; r[1] = q.y;
  }
}
template <typename T>
__device__ __forceinline__ void vst(T* p, const T* r) {
  if constexpr (is_dfl<T>::value) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0].hi, r[0].lo, r[1].hi, r[1].lo);
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
  }
}
template <bool CG, typename T>
__device__ __forceinline__ void vld_global(T* r, const T* p) {
  if constexpr (is_dfl<T>::value) {
    const float4 q = CG ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    r[0] = T(q.x, q.y); r[1] = T(q.z, q.w);
  } else if constexpr (sizeof(T) == 4) {
    const float4 q = CG ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
  } else {
    const double2 q = CG ? __ldcg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
    r[0] = q.x; r[1] = q.y;
  }
}

// out[v] = sum_{m=1..MT} k[m-1] (w[v + D + m - 1 + a] - w[v + D - m + a]) for the
// window w of L values; a = 1 gives d^E (Faraday), a = 0 gives d^B (Ampere).
//
// Compensated values (dfl) take the same taps in the same order with the
// renormalisations deferred: the difference of the two samples is formed by
// TwoSum of the high parts plus the low parts, its product with the tap by
// TwoProd plus the cross terms, and the running sum keeps its error term in a
// separate FP32 accumulator through TwoSum; one renormalisation at the end.
// About 20 FP32 operations per tap; the result is within a few 2^-48 of the
// sum of |k_m| |samples|.
template <typename T, int V, int MT, int D, int L, int A>
__host__ __device__ __forceinline__ void x1_stencil(T* out, const T* row, const T* k) {
  T w[L];
#pragma unroll
  for (int t = 0; t < L; t += V) vld(w + t, row + t);
  if constexpr (is_dfl<T>::value) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int m = 1; m <= MT; ++m) {
        const dfl a = w[v + D + m - 1 + A], b = w[v + D - m + A];
        const dfl d = two_sum(a.hi, -b.hi);
        const float dl = d.lo + (a.lo - b.lo);
        const float p = mul_rn(k[m - 1].hi, d.hi);
        float pe = fmaf(k[m - 1].hi, d.hi, -p);
        pe = fmaf(k[m - 1].hi, dl, pe);
        pe = fmaf(k[m - 1].lo, d.hi, pe);
        const dfl s = two_sum(sh, p);
        sh = s.hi;
        sl += s.lo + pe;
      }
      out[v] = fast_two_sum(sh, sl);
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T acc = 0;
#pragma unroll
      for (int m = 1; m <= MT; ++m) acc += k[m - 1] * (w[v + D + m - 1 + A] - w[v + D - m + A]);
      out[v] = acc;
    }
  }
}

// Faraday over the B region, then Ampere over the tile; writes E^{n+1}, B^{n+1/2}.
// j may be null (no current); with zero_j the tile's current is cleared once read.
// sJ (nullable): the tile's J already staged in shared memory, component-major
// rows of TX values; otherwise J is read from j.  TX is a multiple of V.
template <bool CG, typename T, int NDIM, int MT>
__device__ __forceinline__ void tile_compute(T* const* j, T* const* eo, T* const* bo, FieldDims dim,
                                             const StencilArgs<T>& s, T dt, int TX, int TY, int TZ,
                                             const TileGeom& G, T* sm, bool zero_j,
                                             const T* sJ = nullptr) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach R(MT, V);
  const int n1 = dim.n1, n2 = dim.n2, n3 = (NDIM == 3) ? dim.n3 : 1;
  T* sE = sm;
  T* sB = sm + 3 * G.nE;
  const int nE = G.nE, nB = G.nB;
  const int sE2 = G.WE, sE3 = G.WE * G.WE2;
  const int sB2 = G.WB, sB3 = G.WB * G.WB2;
  const T* E1 = sE;
  const T* E2 = sE + nE;
  const T* E3 = sE + 2 * nE;

  // Faraday: B^{n+1/2} = B^{n-1/2} - dt curl_E E^n over the whole B region
  const int gpB = G.WB / V;
  for (int q = threadIdx.x; q < G.WB2 * G.WB3 * gpB; q += blockDim.x) {
    const int row = q / gpB, col = (q - row * gpB) * V;
    const int l2 = row % G.WB2, l3 = row / G.WB2;
    const int er = l3 * sE3 + l2 * sE2;   // E row of this B row
    const int ec = er + col + R.DE;       // E at this group's columns
    T dE3[V], dE2[V];
    x1_stencil<T, V, MT, R.DE, R.LE, 1>(dE3, E3 + er + col, s.kE);
    x1_stencil<T, V, MT, R.DE, R.LE, 1>(dE2, E2 + er + col, s.kE);
    T a[V], b_[V], c_[V], d_[V];
    T b1[V], b2[V], b3[V];
    const int bq = row * sB2 + col;
    vld(b1, sB + bq);
    vld(b2, sB + nB + bq);
    vld(b3, sB + 2 * nB + bq);
    vld(a, E3 + ec + sE2);
    vld(b_, E3 + ec);
    vld(c_, E1 + ec + sE2);
    vld(d_, E1 + ec);
    T d2E3[V], d2E1[V], d3E2[V], d3E1[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d2E3[v] = s.y2 * (a[v] - b_[v]);
      d2E1[v] = s.y2 * (c_[v] - d_[v]);
      d3E2[v] = 0;
      d3E1[v] = 0;
    }
    if (NDIM == 3) {
      vld(a, E2 + ec + sE3);
      vld(b_, E2 + ec);
      vld(c_, E1 + ec + sE3);
      vld(d_, E1 + ec);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        d3E2[v] = s.y3 * (a[v] - b_[v]);
        d3E1[v] = s.y3 * (c_[v] - d_[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      b1[v] -= d2E3[v] - d3E2[v];   // B1 -= dt (d2 E3 - d3 E2)
      b2[v] -= d3E1[v] - dE3[v];    // B2 -= dt (d3 E1 - d^E1 E3)
      b3[v] -= dE2[v] - d2E1[v];    // B3 -= dt (d^E1 E2 - d2 E1)
    }
    vst(sB + bq, b1);
    vst(sB + nB + bq, b2);
    vst(sB + 2 * nB + bq, b3);
  }
  __syncthreads();

  // Ampere: E^{n+1} = E^n + dt (curl_B B^{n+1/2} - J) over the tile
  const T* B1 = sB;
  const T* B2 = sB + nB;
  const T* B3 = sB + 2 * nB;
  const int TZe = (NDIM == 3) ? TZ : 1;
  const int gpT = TX / V;
  // vector global access: rows start on 16-byte boundaries and so do the arrays
  uintptr_t am = 0;
  for (int c = 0; c < 3; ++c) {
    am |= (uintptr_t)eo[c] | (uintptr_t)bo[c];
    if (j) am |= (uintptr_t)j[c];
  }
  const bool vec_out = (n1 % V) == 0 && (am & 15u) == 0;
  for (int q = threadIdx.x; q < TY * TZe * gpT; q += blockDim.x) {
    const int row = q / gpT, oc = (q - row * gpT) * V;
    const int o2 = row % TY, o3 = row / TY;
    const int gj = G.j0 + o2, gk = G.k0 + o3, gi = G.i0 + oc;
    if (gj >= n2 || (NDIM == 3 && gk >= n3) || gi >= n1) continue;
    const int br = (NDIM == 3 ? (o3 + 1) * sB3 : 0) + (o2 + 1) * sB2;  // B row of this E row
    const int bc = br + oc + R.DB;
    const int ec = (NDIM == 3 ? (o3 + 1) * sE3 : 0) + (o2 + 1) * sE2 + oc + R.DB + R.DE;
    T dB3[V], dB2[V];
    x1_stencil<T, V, MT, R.DB, R.LB, 0>(dB3, B3 + br + oc, s.kB);
    x1_stencil<T, V, MT, R.DB, R.LB, 0>(dB2, B2 + br + oc, s.kB);
    T b1[V], b2[V], b3[V], b1m[V], b3m[V];
    vld(b1, B1 + bc);
    vld(b2, B2 + bc);
    vld(b3, B3 + bc);
    vld(b1m, B1 + bc - sB2);
    vld(b3m, B3 + bc - sB2);
    T d2B3[V], d2B1[V], d3B2[V], d3B1[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d2B3[v] = s.y2 * (b3[v] - b3m[v]);
      d2B1[v] = s.y2 * (b1[v] - b1m[v]);
      d3B2[v] = 0;
      d3B1[v] = 0;
    }
    if (NDIM == 3) {
      T b2k[V], b1k[V];
      vld(b2k, B2 + bc - sB3);
      vld(b1k, B1 + bc - sB3);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        d3B2[v] = s.y3 * (b2[v] - b2k[v]);
        d3B1[v] = s.y3 * (b1[v] - b1k[v]);
      }
    }
    T j1[V], j2[V], j3[V], e1[V], e2[V], e3[V];
    const int64_t gidx = ((int64_t)gk * n2 + gj) * n1 + gi;
    const int nv = min(V, n1 - gi);
    if (sJ) {
      const int jq = row * TX + oc, nJ = TX * TY * TZe;
      vld(j1, sJ + jq);
      vld(j2, sJ + nJ + jq);
      vld(j3, sJ + 2 * nJ + jq);
    } else if (j && vec_out) {
      vld_global<CG>(j1, j[0] + gidx);
      vld_global<CG>(j2, j[1] + gidx);
      vld_global<CG>(j3, j[2] + gidx);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const bool in = j && v < nv;
        j1[v] = in ? gload<CG>(j[0] + gidx + v) : (T)0;
        j2[v] = in ? gload<CG>(j[1] + gidx + v) : (T)0;
        j3[v] = in ? gload<CG>(j[2] + gidx + v) : (T)0;
      }
    }
    vld(e1, E1 + ec);
    vld(e2, E2 + ec);
    vld(e3, E3 + ec);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      e1[v] = e1[v] + ((d2B3[v] - d3B2[v]) - dt * j1[v]);
      e2[v] = e2[v] + ((d3B1[v] - dB3[v]) - dt * j2[v]);
      e3[v] = e3[v] + ((dB2[v] - d2B1[v]) - dt * j3[v]);
    }
    if (vec_out) {
      vst(eo[0] + gidx, e1);
      vst(eo[1] + gidx, e2);
      vst(eo[2] + gidx, e3);
      vst(bo[0] + gidx, b1);
      vst(bo[1] + gidx, b2);
      vst(bo[2] + gidx, b3);
      if (j && zero_j) {
        const T z[V] = {};
        vst(j[0] + gidx, z);
        vst(j[1] + gidx, z);
        vst(j[2] + gidx, z);
      }
    } else {
      for (int v = 0; v < nv; ++v) {
        eo[0][gidx + v] = e1[v];
        eo[1][gidx + v] = e2[v];
        eo[2][gidx + v] = e3[v];
        bo[0][gidx + v] = b1[v];
        bo[1][gidx + v] = b2[v];
        bo[2][gidx + v] = b3[v];
        if (j && zero_j) {
          j[0][gidx + v] = (T)0;
          j[1][gidx + v] = (T)0;
          j[2][gidx + v] = (T)0;
        }
      }
    }
  }
}

// Update tile number `tile` (x1 fastest over ceil(n/T) tiles per axis) with
// synchronous staging.  smem holds field_tile_smem_elems(...) values of T.
template <typename T, int NDIM, bool CG, int MT>
__device__ __forceinline__ void field_tile(const T* const* e, const T* const* b, T* const* j,
                                           T* const* eo, T* const* bo, FieldDims dim,
                                           const StencilArgs<T>& s, T dt, int TX, int TY, int TZ,
                                           int tile, T* sm, bool zero_j = false) {
  const TileGeom G = tile_geom<T, NDIM, MT>(dim, TX, TY, TZ, tile);
  tile_stage_sync<CG, T, NDIM>(e, b, dim, G, sm);
  __syncthreads();
  tile_compute<CG, T, NDIM, MT>(j, eo, bo, dim, s, dt, TX, TY, TZ, G, sm, zero_j);
}

// ---------------------------------------------------------------------------
// TMA staging: one elected thread issues 1D bulk copies (cp.async.bulk) of the
// region rows, completing on an mbarrier that all threads then wait on.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ long long gtimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity; false if it did not complete within
// limit_ns (the caller then reports an error instead of spinning on).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit_ns) {
  const long long t0 = gtimer_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer_ns() - t0 > limit_ns) return false;
  }
}

// Element-wise asynchronous copies (cp.async, 4 or 8 bytes) for rows that bulk
// copies cannot take (row pitch not a multiple of 16 bytes): each lane copies
// W values of a periodic grid row from column c0 into dst, then makes the
// mbarrier track its copies (the pending count rises at issue and falls when
// the copies land; a plain arrival by one thread completes the phase).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src),
               "n"((int)sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_track(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
template <typename T>
__device__ __forceinline__ void async_row(T* dst, const T* row, int c0, int W, int n1, int lane) {
  if (c0 >= 0 && c0 + W <= n1) {
    for (int l = lane; l < W; l += 32) cp_async_elem(dst + l, row + c0 + l);
  } else {
    for (int l = lane; l < W; l += 32) cp_async_elem(dst + l, row + pwrap(c0 + l, n1));
  }
}

// A tile is staged by bulk copies when each region row fits in one grid row
// (a row that crosses the periodic x1 seam is copied in two pieces) and the
// tile is whole (no ragged edge), so its J rows are whole too.  Row starts are
// 16-byte aligned by the caller's check that n1 and TX are multiples of V.
template <typename T, int NDIM>
__device__ __forceinline__ bool tile_tma_ok(FieldDims dim, const TileGeom& G, int TX, int TY,
                                            int TZ) {
  return G.WE <= dim.n1 && G.i0 + TX <= dim.n1 && G.j0 + TY <= dim.n2 &&
         (NDIM == 2 || G.k0 + TZ <= dim.n3);
}

// W values of a periodic grid row from column c0 (|c0| < n1, W <= n1), in at
// most two bulk copies
template <typename T>
__device__ __forceinline__ void bulk_row(T* dst, const T* row, int c0, int W, int n1,
                                         uint64_t* bar) {
  const int s0 = c0 < 0 ? c0 + n1 : (c0 >= n1 ? c0 - n1 : c0);
  const int w1 = min(W, n1 - s0);
  bulk_g2s(dst, row + s0, (uint32_t)(w1 * sizeof(T)), bar);
  if (w1 < W) bulk_g2s(dst + w1, row, (uint32_t)((W - w1) * sizeof(T)), bar);
}

// one warp: lane 0 arms the barrier with the byte count, then the lanes issue
// the region rows (and, with j, the tile's J rows into sJ)
template <typename T, int NDIM>
__device__ __forceinline__ void tile_stage_tma(const T* const* e, const T* const* b,
                                               const T* const* j, FieldDims dim, const TileGeom& G,
                                               int TX, int TY, int TZ, T* sm, T* sJ, uint64_t* bar,
                                               int lane) {
  const int n1 = dim.n1, n2 = dim.n2, n3 = (NDIM == 3) ? dim.n3 : 1;
  const int nrE = 3 * G.WE2 * G.WE3, nrB = 3 * G.WB2 * G.WB3;
  const int TZe = (NDIM == 3) ? TZ : 1;
  const int nrJ = j ? 3 * TY * TZe : 0;
  if (lane == 0)
    mbar_expect_tx(bar, (uint32_t)(((int64_t)nrE * G.WE + (int64_t)nrB * G.WB + (int64_t)nrJ * TX) *
                                   sizeof(T)));
  __syncwarp();
  T* sE = sm;
  T* sB = sm + 3 * G.nE;
  for (int row = lane; row < nrJ; row += 32) {
    const int o2 = row % TY, r = row / TY;
    const int o3 = r % TZe, c = r / TZe;
    bulk_g2s(sJ + row * TX, j[c] + ((int64_t)(G.k0 + o3) * n2 + (G.j0 + o2)) * n1 + G.i0,
             (uint32_t)(TX * sizeof(T)), bar);
  }
  for (int row = lane; row < nrE; row += 32) {
    const int l2 = row % G.WE2, r = row / G.WE2;
    const int l3 = r % G.WE3, c = r / G.WE3;
    const int gj = pwrap(G.j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(G.k0 - 1 + l3, n3) : 0;
    bulk_row(sE + row * G.WE, e[c] + ((int64_t)gk * n2 + gj) * n1, G.Es, G.WE, n1, bar);
  }
  for (int row = lane; row < nrB; row += 32) {
    const int l2 = row % G.WB2, r = row / G.WB2;
    const int l3 = r % G.WB3, c = r / G.WB3;
    const int gj = pwrap(G.j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(G.k0 - 1 + l3, n3) : 0;
    bulk_row(sB + row * G.WB, b[c] + ((int64_t)gk * n2 + gj) * n1, G.Bs, G.WB, n1, bar);
  }
}

// shared-memory values one tile's E and B regions need
__host__ __device__ inline size_t field_tile_smem_elems(int ndim, int TX, int TY, int TZ, int M,
                                                        int tsize) {
  const int V = 16 / tsize;
  const Reach R(stencil_mt(M), V);
  const size_t nE = (size_t)R.WE(TX, V) * (TY + 2) * (ndim == 3 ? TZ + 2 : 1);
  const size_t nB = (size_t)R.WB(TX, V) * (TY + 1) * (ndim == 3 ? TZ + 1 : 1);
  return 3 * (nE + nB);
}

}  // namespace pic
