// particle_kernels.cuh -- the tiled particle kernel, the time-centred-B row
// kernel and the straggler kernel of libpic with their launchers, as templates
// over the field type; particles_f32.cu, particles_f64.cu and particles_dfl.cu
// instantiate one field type each (parallel compilation).
//
// Particles are binned by tile (a box of cells).  A row pass first forms the
// time-centred B^n = B^{n-1/2} - (dt/2) d_E x E^n (Eq. (7) in its half-step form)
// over the grid.  One CTA owns one tile: it stages E^n and B^n of the tile plus
// a guard in shared memory and runs every particle of the bin through
//   gather (App. A, quadratic B-spline at each component's staggered node)
//   -> push (Boris, Higuera-Cary or analytic, FP64)
//   -> x^{n+1} = x^n + dt u/gamma (FP64)
//   -> Esirkepov deposit (Sec. 3.3) into a shared-memory current window (int32
//      fixed point),
// then adds the window into the global current once.  Bins are rebuilt every
// few steps; a particle that has drifted out of its tile's window takes the
// global-memory path of straggler_kernel instead, so correctness never depends
// on the rebinning interval.
#pragma once
#include <math.h>

#include "common.cuh"
#include "field_tile.cuh"
#include "particle_core.cuh"

namespace pic {

namespace {

// Visit every row (c, l3, l2), c < 3, l3 < N3, l2 < N2, of a window whose rows
// hold W1 values, spread over the CTA's warps by nested loops (no integer
// division per row); rows of at most 16 values go two per warp, 16 lanes each.
// (3D windows: short rows and few particles per tile, so this bookkeeping
// would otherwise dominate the tile's instructions.)
// f(c, l2, l3, sub_lane, lanes_per_row) runs on the lanes of one row.
template <class F>
__device__ __forceinline__ void for_window_rows(int N2, int N3, int W1, int lane, int warp,
                                                int nwarp, F&& f) {
  const int split = W1 <= 16 ? 2 : 1;
  const int sw = 32 / split;
  const int sub = split == 2 ? lane >> 4 : 0, sl = split == 2 ? lane & 15 : lane;
  const int step = nwarp * split;
  for (int c = 0; c < 3; ++c)
    for (int l3 = 0; l3 < N3; ++l3)
      for (int l2 = warp * split + sub; l2 < N2; l2 += step) f(c, l2, l3, sl, sw);
}

// W values of a periodic row from column g0, lanes sl of sw per row
template <typename T>
__device__ __forceinline__ void stage_row_lanes(T* dst, const T* src, int g0, int W, int n1, int sl,
                                                int sw) {
  if (g0 >= 0 && g0 + W <= n1) {
    for (int l1 = sl; l1 < W; l1 += sw) dst[l1] = src[g0 + l1];
  } else {
    for (int l1 = sl; l1 < W; l1 += sw) dst[l1] = src[pwrap(g0 + l1, n1)];
  }
}

// threads 0 .. NDIM+3 ask L2 for one particle array each over [c0, c1) (bulk
// prefetch: 16-byte aligned start and size, so the range is cut to even indices)
template <int NDIM>
__device__ __forceinline__ void prefetch_chunk(const PartPtrs& p, int64_t c0, int64_t c1) {
  const int t = threadIdx.x;
  if (t >= NDIM + 4) return;
  const int64_t s0 = c0 & ~1LL, e0 = c1 & ~1LL;
  if (e0 <= s0) return;
  const int c = t - NDIM;   // constant indices only: the pointer arrays stay in the parameter bank
  const double* arr = t < NDIM ? (t == 0 ? p.x[0] : (t == 1 ? p.x[1] : p.x[2]))
                               : (c == 0 ? p.u[0] : (c == 1 ? p.u[1] : (c == 2 ? p.u[2] : p.w)));
  if ((reinterpret_cast<uintptr_t>(arr) & 15u) != 0) return;   // a hint only: skip if unaligned
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(arr + s0),
               "r"((unsigned)((e0 - s0) * 8)) : "memory");
}

// The time-centred B^n is read from a global array formed once per step by
// bbar_rows_kernel; E^n and B^n are staged over the particle window, the
// current is accumulated in a shared-memory window (in int32 fixed point,
// FixAcc / FixAcc64) and added into the global current once.
// All staging and the current flush run row by row, one warp per row.
// PUSH: the pusher, fixed per instance so that the 2D mixed-precision Boris
// kernel is not held to the analytic pusher's register budget: it fits in 64
// registers and runs 4 CTAs per SM instead of 3.  8-byte fields: the windows
// fit 2 (2D) or 1 (3D) CTAs per SM, so the register budget follows.
template <typename T, int NDIM, int PUSH, bool GAIN>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? ((PUSH == PIC_BORIS && NDIM == 2) ? 4 : 3)
                                                      : (NDIM == 2 ? 2 : 1))
    particle_kernel(FieldPtrs<T> f, BbarPtrs<T> bg, PartPtrs p, GridArgs g, StencilArgs<T> s,
                    PartTile t, PartArgs a, BinBufs bins) {
  using D = typename DepositOf<T>::type;
  // current window: FP32 deposits as two int32 fixed-point sums (FixAcc), FP64
  // deposits as three (FixAcc64)
  constexpr bool F64 = std::is_same<D, double>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long wmax_warp[32];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int64_t tile = blockIdx.x;
  const int64_t pbeg = bins.start[tile], pend = bins.start[tile + 1];
  if (pbeg == pend) return;
  prefetch_chunk<NDIM>(p, pbeg, min(pend, pbeg + (int64_t)blockDim.x));
  int tc[3];
  {
    int64_t r = tile;
    tc[0] = (int)(r % t.nt[0]);
    r /= t.nt[0];
    tc[1] = (int)(r % t.nt[1]);
    tc[2] = (int)(r / t.nt[1]);
  }
  const int n1 = g.n[0], n2 = g.n[1], n3 = (NDIM == 3) ? g.n[2] : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // window: the tile plus g - 1 guard cells below and g above (a particle's
  // gather and deposit reach two nodes below its cell and three above; g - 3
  // cells of drift are allowed on both sides)
  int W[3], wlo[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    W[d] = (d < NDIM) ? t.t[d] + 2 * t.g[d] - 1 : 1;
    wlo[d] = (d < NDIM) ? tc[d] * t.t[d] - (t.g[d] - 1) : 0;
  }
  const int nW = W[0] * W[1] * W[2];
  T* sE = sm;                 // [3][W3][W2][W1]
  T* sB = sE + 3 * nW;        // [3][W3][W2][W1], the time-centred B
  int* sJh = reinterpret_cast<int*>(sB + 3 * nW);   // current: [3][W3][W2][W1] per limb, hi first
  int* sJl = sJh + 3 * nW;
  int* sJc = sJl + 3 * nW;                          // FP64: the third limb

  {
    // largest |w| of the tile (non-negative doubles order as their bit patterns)
    unsigned long long wm = 0ull;
    for (int64_t q = pbeg + threadIdx.x; q < pend; q += blockDim.x)
      wm = max(wm, (unsigned long long)__double_as_longlong(p.w[q]) & 0x7fffffffffffffffull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    if (lane == 0) wmax_warp[warp] = wm;
  }
  if constexpr (NDIM == 3) {
    // short rows: division-free row loops, two rows per warp
    for_window_rows(W[1], W[2], W[0], lane, warp, nwarp, [&](int c, int l2, int l3, int sl, int sw) {
      const int gj = pwrap(wlo[1] + l2, n2);
      const int gk = pwrap(wlo[2] + l3, n3);
      const int64_t r = ((int64_t)gk * n2 + gj) * n1;
      const int o = ((c * W[2] + l3) * W[1] + l2) * W[0];
      const T* e = c == 0 ? f.e[0] : (c == 1 ? f.e[1] : f.e[2]);
      const T* b = c == 0 ? bg.b[0] : (c == 1 ? bg.b[1] : bg.b[2]);
      stage_row_lanes(sE + o, e + r, wlo[0], W[0], n1, sl, sw);
      stage_row_lanes(sB + o, b + r, wlo[0], W[0], n1, sl, sw);
    });
  } else {
    for (int row = warp; row < 3 * W[1]; row += nwarp) {
      const int l2 = row % W[1], c = row / W[1];
      const int64_t r = (int64_t)pwrap(wlo[1] + l2, n2) * n1;
      stage_row<false>(sE + row * W[0], f.e[c] + r, wlo[0], W[0], n1, lane);
      stage_row<false>(sB + row * W[0], bg.b[c] + r, wlo[0], W[0], n1, lane);
    }
  }
  for (int q = threadIdx.x; q < (F64 ? 9 : 6) * nW; q += blockDim.x) sJh[q] = 0;
  __syncthreads();
  float S = 1.0f, L = 1.0f;
  int eS = 0, l64 = 0;
  {
    unsigned long long wm = 0ull;
    for (int k = 0; k < nwarp; ++k) wm = max(wm, wmax_warp[k]);
    // |contribution| <= |w|: a J_d term is -w (dx_d/dt) times a difference of the
    // cumulative shape weights before and after the move (at most |delta_d| in
    // magnitude: the node sums of the quadratic spline have slope <= 1) times a
    // time-averaged shape weight (<= 1), so at most |w| |v_d| < |w|; the 2D
    // out-of-plane term is w v3 times a path-averaged weight product (<= 1)
    if constexpr (F64) fix64_scales(pend - pbeg, __longlong_as_double((long long)wm), eS, l64);
    else fix_scales(pend - pbeg, narrow_signed(__longlong_as_double((long long)wm)) * 1.001f, S, L);
  }

  SmemView<T> ve[3], vb[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ve[c] = SmemView<T>{sE + c * nW, W[0], W[0] * W[1], 0};
    vb[c] = SmemView<T>{sB + c * nW, W[0], W[0] * W[1], 0};
  }
  using Acc = typename std::conditional<F64, FixAcc64, FixAcc>::type;
  Acc acc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if constexpr (F64)
      acc[c] = FixAcc64{sJh + c * nW, sJl + c * nW, sJc + c * nW, W[0], W[0] * W[1], eS, l64};
    else acc[c] = FixAcc{sJh + c * nW, sJl + c * nW, W[0], W[0] * W[1], S, L};
  }
  const float invS = 1.0f / S, invSL = 1.0f / (S * L);   // powers of two: exact
  // FP64 limb weights 2^-eS, 2^-(eS + l), 2^-(eS + 2l), from the exponent bits
  auto pow2 = [](int e) { return __longlong_as_double((long long)(uint64_t)(1023 + e) << 52); };
  const double i0 = F64 ? pow2(-eS) : 0.0, i1 = F64 ? pow2(-eS - l64) : 0.0,
               i2 = F64 ? pow2(-eS - 2 * l64) : 0.0;
  // value of window node q of component c
  auto jval = [&](int c, int q) -> D {
    if constexpr (F64) return fix64_decode(sJh[c * nW + q], sJl[c * nW + q], sJc[c * nW + q], i0, i1, i2);
    else return fix_decode(sJh[c * nW + q], sJl[c * nW + q], invS, invSL);
  };
  int ulo[3], uhi[3];   // periodic unwrap limits of the window-local node index
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ulo[d] = (W[d] - g.n[d]) / 2;
    uhi[d] = ulo[d] + g.n[d];
  }
  for (int64_t q = pbeg + threadIdx.x; q < pend; q += blockDim.x) {
    {
      const int64_t c0 = q - threadIdx.x + blockDim.x;
      if (c0 < pend) prefetch_chunk<NDIM>(p, c0, min(pend, c0 + (int64_t)blockDim.x));
    }
    int li[3], gc[3];
    T fr[3];
    bool inside = true;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const double c = p.x[d][q] * g.inv_dx[d];
      double frac;
      gc[d] = floor_split(c, frac);             // exact floor and fraction, no FP64 conversion
      fr[d] = to_prec<T>(frac);
      int l = gc[d] - wlo[d];
      if (l < ulo[d]) l += g.n[d];
      else if (l >= uhi[d]) l -= g.n[d];
      li[d] = l;
      inside = inside && l >= 2 && l <= W[d] - 4;
    }
    if (!inside) {
      const unsigned long long slot = atomicAdd(bins.strag_count, 1ull);
      bins.strag[slot] = q;
      continue;
    }
    advance_particle<T, NDIM, PUSH, GAIN>(ve, vb, acc, p, q, li, fr, gc, g, a, bins.err);
  }
  __syncthreads();
  if constexpr (NDIM == 3) {
    for_window_rows(W[1], W[2], W[0], lane, warp, nwarp, [&](int c, int l2, int l3, int sl, int sw) {
      const int gj = pwrap(wlo[1] + l2, n2);
      const int gk = pwrap(wlo[2] + l3, n3);
      T* dst = (c == 0 ? f.j[0] : (c == 1 ? f.j[1] : f.j[2])) + ((int64_t)gk * n2 + gj) * n1;
      const int o = (l3 * W[1] + l2) * W[0];
      const bool inrow = wlo[0] >= 0 && wlo[0] + W[0] <= n1;
      for (int l1 = sl; l1 < W[0]; l1 += sw) {
        const D v = jval(c, o + l1);
        if (v != (D)0) atomic_acc(dst + (inrow ? wlo[0] + l1 : pwrap(wlo[0] + l1, n1)), v);
      }
    });
  } else {
    for (int row = warp; row < 3 * W[1]; row += nwarp) {
      const int l2 = row % W[1], c = row / W[1];
      const int gj = pwrap(wlo[1] + l2, n2);
      T* dst = f.j[c] + (int64_t)gj * n1;
      for (int l1 = lane; l1 < W[0]; l1 += 32) {
        const D v = jval(c, l2 * W[0] + l1);
        if (v != (D)0) atomic_acc(dst + pwrap(wlo[0] + l1, n1), v);
      }
    }
  }
}

// Time-centred B^n = B^{n-1/2} - (dt/2) d_E x E^n into bg, one x1 row segment of
// kBbarT * V cells per CTA, V = 16/sizeof(T) consecutive outputs per thread: the
// E2/E3 rows it differentiates along x1 are staged with the stencil's reach and
// differentiated by the register-blocked x1 stencil of the field kernels (the
// same taps in the same order as the plain sum over m = 1..M).
constexpr int kBbarT = 256;

template <typename T, int NDIM, int MT>
__global__ void __launch_bounds__(kBbarT) bbar_rows_kernel(FieldPtrs<T> f, BbarPtrs<T> bg, GridArgs g,
                                                           StencilArgs<T> s) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int TXV = kBbarT * V;
  const int n1 = g.n[0], n2 = g.n[1], n3 = (NDIM == 3) ? g.n[2] : 1;
  const int nseg = (n1 + TXV - 1) / TXV;
  const int seg = blockIdx.x % nseg;
  const int64_t row = blockIdx.x / nseg;
  const int j = (int)(row % n2), k = (int)(row / n2);
  const int i0 = seg * TXV;
  const int WL = TXV - V + RC.LE;   // staged values per row, from column i0 - DE
  T* s2 = sm;                       // E2 row
  T* s3 = sm + ceil_to(WL, V);      // E3 row
  const int64_t r0 = ((int64_t)k * n2 + j) * n1;
  for (int l = threadIdx.x; l < WL; l += blockDim.x) {
    const int gi = pwrap(i0 - RC.DE + l, n1);
    s2[l] = f.e[1][r0 + gi];
    s3[l] = f.e[2][r0 + gi];
  }
  __syncthreads();
  const int col = threadIdx.x * V;
  if (i0 + col >= n1) return;
  T dE3[V], dE2[V];
  x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE3, s3 + col, s.kE);
  x1_stencil<T, V, MT, RC.DE, RC.LE, 1>(dE2, s2 + col, s.kE);
  const int64_t q0 = r0 + i0 + col;
  const int64_t dj = (int64_t)(j + 1 == n2 ? 0 : j + 1) * n1 - (int64_t)j * n1;
  const int64_t dk = NDIM == 3 ? ((int64_t)(k + 1 == n3 ? 0 : k + 1) - k) * n2 * n1 : 0;
  auto out = [&](int v, T e1, T e1j, T e1k, T e2, T e2k, T e3, T e3j, T b1, T b2, T b3, T* o) {
    const T d2E3 = s.y2 * (e3j - e3);
    const T d2E1 = s.y2 * (e1j - e1);
    T d3E2 = 0, d3E1 = 0;
    if (NDIM == 3) {
      d3E2 = s.y3 * (e2k - e2);
      d3E1 = s.y3 * (e1k - e1);
    }
    o[0] = b1 - (T)0.5 * (d2E3 - d3E2);
    o[1] = b2 - (T)0.5 * (d3E1 - dE3[v]);
    o[2] = b3 - (T)0.5 * (dE2[v] - d2E1);
  };
  if (n1 % V == 0 && i0 + col + V <= n1) {
    // whole aligned group: 16-byte loads and stores
    T e1[V], e1j[V], e1k[V], e2[V], e2k[V], e3[V], e3j[V], b1[V], b2[V], b3[V];
    vld_global<false>(e1, f.e[0] + q0);
    vld_global<false>(e1j, f.e[0] + q0 + dj);
    vld_global<false>(e2, f.e[1] + q0);
    vld_global<false>(e3, f.e[2] + q0);
    vld_global<false>(e3j, f.e[2] + q0 + dj);
    if (NDIM == 3) {
      vld_global<false>(e1k, f.e[0] + q0 + dk);
      vld_global<false>(e2k, f.e[1] + q0 + dk);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) e1k[v] = e2k[v] = (T)0;
    }
    vld_global<false>(b1, f.b[0] + q0);
    vld_global<false>(b2, f.b[1] + q0);
    vld_global<false>(b3, f.b[2] + q0);
    T o1[V], o2[V], o3[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T o[3];
      out(v, e1[v], e1j[v], e1k[v], e2[v], e2k[v], e3[v], e3j[v], b1[v], b2[v], b3[v], o);
      o1[v] = o[0];
      o2[v] = o[1];
      o3[v] = o[2];
    }
    vst(bg.b[0] + q0, o1);
    vst(bg.b[1] + q0, o2);
    vst(bg.b[2] + q0, o3);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (i0 + col + v >= n1) break;
      const int64_t q = q0 + v;
      T o[3];
      out(v, f.e[0][q], f.e[0][q + dj], NDIM == 3 ? f.e[0][q + dk] : (T)0, f.e[1][q],
          NDIM == 3 ? f.e[1][q + dk] : (T)0, f.e[2][q], f.e[2][q + dj], f.b[0][q], f.b[1][q],
          f.b[2][q], o);
      bg.b[0][q] = o[0];
      bg.b[1][q] = o[1];
      bg.b[2][q] = o[2];
    }
  }
}

template <typename T, int NDIM, int MT>
cudaError_t launch_bbar_rows(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const GridArgs& g,
                             const StencilArgs<T>& s, cudaStream_t st) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  const int TXV = kBbarT * V;
  const size_t smem = 2 * (size_t)ceil_to(TXV - V + RC.LE, V) * sizeof(T);
  const int64_t nb = (int64_t)((g.n[0] + TXV - 1) / TXV) * g.n[1] * (NDIM == 3 ? g.n[2] : 1);
  bbar_rows_kernel<T, NDIM, MT><<<(unsigned)nb, kBbarT, smem, st>>>(f, bg, g, s);
  return cudaGetLastError();
}

template <typename T, int NDIM>
cudaError_t launch_bbar_rows_mt(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const GridArgs& g,
                                const StencilArgs<T>& s, cudaStream_t st) {
  switch (stencil_mt(s.M)) {
    case 8: return launch_bbar_rows<T, NDIM, 8>(f, bg, g, s, st);
    case 16: return launch_bbar_rows<T, NDIM, 16>(f, bg, g, s, st);
    default: return launch_bbar_rows<T, NDIM, 32>(f, bg, g, s, st);
  }
}

// Particles that left their tile's window: the whole update through global
// memory, with the time-centred B from bg (formed by the tile step's launcher).
template <typename T, int NDIM, bool GAIN>
__global__ void straggler_kernel(FieldPtrs<T> f, BbarPtrs<T> bg, PartPtrs p, GridArgs g,
                                 StencilArgs<T> s, PartArgs a, BinBufs bins) {
  (void)s;
  const unsigned long long cnt = *bins.strag_count;
  const int n1 = g.n[0], n2 = g.n[1], n3 = (NDIM == 3) ? g.n[2] : 1;
  GlobView<T> ve[3], vb[3];
  GlobAcc<T> acc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ve[c] = GlobView<T>{f.e[c], n1, n2, n3, n1};
    vb[c] = GlobView<T>{bg.b[c], n1, n2, n3, n1};
    acc[c] = GlobAcc<T>{f.j[c], n1, n2, n3, n1};
  }
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cnt;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t q = bins.strag[i];
    int li[3];
    T fr[3];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const double c = p.x[d][q] * g.inv_dx[d];
      double frac;
      li[d] = floor_split(c, frac);
      fr[d] = to_prec<T>(frac);
    }
    advance_particle<T, NDIM, -1, GAIN>(ve, vb, acc, p, q, li, fr, li, g, a, bins.err);
  }
}

}  // namespace

// one CTA per particle tile
template <typename T, class K>
cudaError_t launch_tiles(K kern, const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                         const GridArgs& g, const StencilArgs<T>& s, const PartTile& t,
                         const PartArgs& a, const BinBufs& b, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)t.ntiles, 256, smem, st>>>(f, bg, p, g, s, t, a, b);
  return cudaGetLastError();
}

// the tile kernel instance of the context's pusher
template <typename T, int NDIM, bool GAIN>
cudaError_t launch_pushers(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                           const GridArgs& g, const StencilArgs<T>& s, const PartTile& t,
                           const PartArgs& a, const BinBufs& b, size_t smem, cudaStream_t st) {
  if (a.pusher == PIC_ANALYTIC)
    return launch_tiles(particle_kernel<T, NDIM, PIC_ANALYTIC, GAIN>, f, bg, p, g, s, t, a, b, smem,
                        st);
  if (a.pusher == PIC_HC)
    return launch_tiles(particle_kernel<T, NDIM, PIC_HC, GAIN>, f, bg, p, g, s, t, a, b, smem, st);
  return launch_tiles(particle_kernel<T, NDIM, PIC_BORIS, GAIN>, f, bg, p, g, s, t, a, b, smem, st);
}

template <typename T>
cudaError_t launch_particle_step(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                                 const GridArgs& g, const StencilArgs<T>& s, const PartTile& t,
                                 const PartArgs& a, const BinBufs& b, cudaStream_t st) {
  const size_t smem = particle_smem_bytes(g.ndim, sizeof(T), t, s.M);
  cudaError_t e;
  if (!a.bbar_ready) {
    // form the time-centred B once for the whole grid, then the tiles read it
    // (with the spectral field path it is already in bg)
    e = g.ndim == 3 ? launch_bbar_rows_mt<T, 3>(f, bg, g, s, st) : launch_bbar_rows_mt<T, 2>(f, bg, g, s, st);
    if (e != cudaSuccess) return e;
  }
  if (g.ndim == 3)
    e = p.wl ? launch_pushers<T, 3, true>(f, bg, p, g, s, t, a, b, smem, st)
             : launch_pushers<T, 3, false>(f, bg, p, g, s, t, a, b, smem, st);
  else
    e = p.wl ? launch_pushers<T, 2, true>(f, bg, p, g, s, t, a, b, smem, st)
             : launch_pushers<T, 2, false>(f, bg, p, g, s, t, a, b, smem, st);
  return e;
}

template <typename T, int NDIM>
void launch_straggler_nd(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                         const GridArgs& g, const StencilArgs<T>& s, const PartArgs& a,
                         const BinBufs& b, cudaStream_t st) {
  if (p.wl) straggler_kernel<T, NDIM, true><<<152, 128, 0, st>>>(f, bg, p, g, s, a, b);
  else straggler_kernel<T, NDIM, false><<<152, 128, 0, st>>>(f, bg, p, g, s, a, b);
}

template <typename T>
cudaError_t launch_straggler_step(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                                  const GridArgs& g, const StencilArgs<T>& s, const PartArgs& a,
                                  const BinBufs& b, int64_t max_count, cudaStream_t st) {
  (void)max_count;
  if (g.ndim == 3) launch_straggler_nd<T, 3>(f, bg, p, g, s, a, b, st);
  else launch_straggler_nd<T, 2>(f, bg, p, g, s, a, b, st);
  return cudaGetLastError();
}

#define PIC_PARTICLE_INST(T)                                                                  \
  template cudaError_t launch_particle_step<T>(const FieldPtrs<T>&, const BbarPtrs<T>&,       \
                                               const PartPtrs&, const GridArgs&,              \
                                               const StencilArgs<T>&, const PartTile&,        \
                                               const PartArgs&, const BinBufs&, cudaStream_t); \
  template cudaError_t launch_straggler_step<T>(const FieldPtrs<T>&, const BbarPtrs<T>&,       \
                                                const PartPtrs&, const GridArgs&,              \
                                                const StencilArgs<T>&, const PartArgs&,        \
                                                const BinBufs&, int64_t, cudaStream_t);

}  // namespace pic
