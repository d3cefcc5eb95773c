// fields.cu -- field kernels of libpic.
//
// field_step: one fused pass per tile of
//   B^{n+1/2} = B^{n-1/2} - dt d_E x E^n          (Eq. (1), App. B Eq. (B.1))
//   E^{n+1}   = E^n + dt (d_B x B^{n+1/2} - J)     (Eq. (1), App. B Eq. (B.2))
// with E^n and B^{n-1/2} staged in shared memory over the tile plus the halo the
// two wide x1 stencils need (2M-1 cells each side in x1, one cell in x2/x3).
// Each value of E, B, J is read from HBM once and E, B written once (15 values
// per cell, the algorithmic minimum); halo re-reads hit L2.
#include <algorithm>

#include "common.cuh"
#include "field_rows.cuh"
#include "field_tile.cuh"

namespace pic {

namespace {

template <typename T>
struct OutPtrs {
  T* e[3];
  T* b[3];
};

template <typename T, int NDIM, int MT>
__global__ void __launch_bounds__(512, 1) field_step_kernel(FieldPtrs<T> f, OutPtrs<T> o, GridArgs g,
                                                         StencilArgs<T> s, int TX, int TY,
                                                         int TZ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FieldDims dim{g.n[0], g.n[1], g.n[2]};
  field_tile<T, NDIM, false, MT>(f.e, f.b, f.j, o.e, o.b, dim, s, (T)g.dt, TX, TY, TZ,
                             (int)blockIdx.x, reinterpret_cast<T*>(smem_raw));
}

// Persistent form: each CTA walks tiles blockIdx.x, +gridDim.x, ... with two
// shared-memory buffers.  While a tile is computed, the next tile's E, B and J
// rows stream into the other buffer as 1D bulk copies completing on an
// mbarrier; tiles at the x1 seam or ragged edges are staged with plain loads.
template <typename T, int NDIM, int MT>
__global__ void __launch_bounds__(512, 1) field_step_tma_kernel(FieldPtrs<T> f, OutPtrs<T> o,
                                                             GridArgs g, StencilArgs<T> s, int TX,
                                                             int TY, int TZ, int ntiles,
                                                             int buf_elems, unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem_tma[];
  const FieldDims dim{g.n[0], g.n[1], g.n[2]};
  const T dt = (T)g.dt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int TZe = (NDIM == 3) ? TZ : 1;
  const int jel = 3 * TX * TY * TZe;  // J values at the end of each buffer
  const long long limit_ns = 2000000000LL;
  // current / next buffer, its mbarrier, phase parity and whether bulk copies fill it
  uint64_t* barc = reinterpret_cast<uint64_t*>(smem_tma);
  uint64_t* barn = barc + 1;
  T* bufc = reinterpret_cast<T*>(smem_tma + 128);
  T* bufn = bufc + buf_elems;
  uint32_t parc = 0u, parn = 0u;
  bool tmac = false, tman = false;
  if (threadIdx.x == 0) {
    mbar_init(barc);
    mbar_init(barn);
    mbar_init_fence();
  }
  __syncthreads();
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  {
    const TileGeom G = tile_geom<T, NDIM, MT>(dim, TX, TY, TZ, tile);
    tmac = tile_tma_ok<T, NDIM>(dim, G, TX, TY, TZ);
    if (tmac) {
      if (warp == 0)
        tile_stage_tma<T, NDIM>(f.e, f.b, f.j, dim, G, TX, TY, TZ, bufc, bufc + buf_elems - jel,
                                barc, lane);
    } else {
      tile_stage_sync<false, T, NDIM>(f.e, f.b, dim, G, bufc);
    }
  }
  for (; tile < ntiles; tile += gridDim.x) {
    bool ok = true;
    if (tmac) {
      ok = mbar_wait(barc, parc, limit_ns);
      parc ^= 1u;
    }
    if (__syncthreads_or(!ok)) {
      // give the copies in flight a last bounded chance to land, then leave
      if (threadIdx.x == 0) atomicOr(err, ERRBIT_TIMEOUT);
      if (tmac) mbar_wait(barc, parc ^ 1u, limit_ns);
      return;
    }
    const int next = tile + gridDim.x;
    TileGeom Gn;
    tman = false;
    if (next < ntiles) {
      Gn = tile_geom<T, NDIM, MT>(dim, TX, TY, TZ, next);
      tman = tile_tma_ok<T, NDIM>(dim, Gn, TX, TY, TZ);
      if (tman && warp == 0)
        tile_stage_tma<T, NDIM>(f.e, f.b, f.j, dim, Gn, TX, TY, TZ, bufn, bufn + buf_elems - jel,
                                barn, lane);
    }
    const TileGeom G = tile_geom<T, NDIM, MT>(dim, TX, TY, TZ, tile);
    tile_compute<false, T, NDIM, MT>(f.j, o.e, o.b, dim, s, dt, TX, TY, TZ, G, bufc, false,
                                 tmac && f.j ? bufc + buf_elems - jel : nullptr);
    // this buffer is written by bulk copies next; order the generic-proxy
    // accesses above before them
    fence_proxy_async();
    if (next < ntiles && !tman) tile_stage_sync<false, T, NDIM>(f.e, f.b, dim, Gn, bufn);
    // the next buffer becomes the current one
    T* tb = bufc; bufc = bufn; bufn = tb;
    uint64_t* tr = barc; barc = barn; barn = tr;
    const uint32_t tp = parc; parc = parn; parn = tp;
    tmac = tman;
  }
}

// 2D rows streamed per warp.  Work item = a strip of SW x1 columns x R rows;
// each warp takes items independently (no CTA barrier) and walks the rows of
// its strip along x2.  Stage q of an item holds the rows t = r0-1+q of E^n and
// B^{n-1/2}, bulk-copied into a ring of NS slots ahead of use; J row t is read
// from global memory into registers before the row's Faraday (it is used once).
// Faraday forms B^{n+1/2} row t from E rows t, t+1 into a two-row ring, then
// Ampere forms E^{n+1} row t from B^{n+1/2} rows t, t-1.  Every B^{n+1/2} value
// is computed once per strip (one extra row per item, no x2 halo
// recomputation) and the x1 halo is the stencils' reach only.

// Column groups per lane whose J the 2D row kernel holds in registers.
constexpr int kMarchJGroups = 3;

struct MarchShape {
  int SW, R, NS, nstrips, nitems;
  int WE, WB, stage_elems, warp_elems, bar_bytes;
};

template <typename T, int MT>
__global__ void __launch_bounds__(512, 1) field_march_kernel(FieldPtrs<T> f, OutPtrs<T> o, GridArgs g,
                                                          StencilArgs<T> s, MarchShape ms,
                                                          unsigned* err) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  extern __shared__ __align__(128) unsigned char smem_m[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n1 = g.n[0], n2 = g.n[1];
  const int SW = ms.SW, NS = ms.NS, WE = ms.WE, WB = ms.WB;
  const T dt = (T)g.dt;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_m) + wib * NS;
  T* wbase = reinterpret_cast<T*>(smem_m + ms.bar_bytes) + (size_t)wib * ms.warp_elems;
  T* bnew = wbase + NS * ms.stage_elems;  // [2 rows][3 components][WB]
  const long long limit_ns = 2000000000LL;
  if (lane == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k]);
    mbar_init_fence();
  }
  __syncwarp();
  const int gw = blockIdx.x * nw + wib, tw = gridDim.x * nw;

  // Issue cursor: item ii (geometry cached), stage iq, ring slot islot.  Stages
  // are waited for in the order they were issued: wslot is the next slot to
  // wait on and bit k of wpar the phase parity its barrier completes next.
  int ii = gw, iq = 0, islot = 0, inflight = 0;
  int ii0 = 0, ir0 = 0, iRr = 0;
  auto item_geom = [&](int it, int& i0, int& r0, int& Rr) {
    const int chunk = it / ms.nstrips;
    i0 = (it - chunk * ms.nstrips) * SW;
    r0 = chunk * ms.R;
    Rr = min(ms.R, n2 - r0);
  };
  if (ii < ms.nitems) item_geom(ii, ii0, ir0, iRr);
  const T* eb[3] = {f.e[0], f.e[1], f.e[2]};
  const T* bb[3] = {f.b[0], f.b[1], f.b[2]};
  const int c3 = lane % 3;
  const T* my_e = c3 == 0 ? eb[0] : (c3 == 1 ? eb[1] : eb[2]);
  const T* my_b = c3 == 0 ? bb[0] : (c3 == 1 ? bb[1] : bb[2]);
  auto issue = [&]() {
    if (ii >= ms.nitems) return;
    T* st = wbase + islot * ms.stage_elems;
    const int t = ir0 - 1 + iq;
    const int gj = t < 0 ? t + n2 : (t >= n2 ? t - n2 : t);
    const bool hasB = iq <= iRr;
    if (lane == 0)
      mbar_expect_tx(&bars[islot], (uint32_t)((3 * WE + (hasB ? 3 * WB : 0)) * sizeof(T)));
    __syncwarp();
    if (lane < 3) {
      bulk_row(st + c3 * WE, my_e + (int64_t)gj * n1, ii0 - RC.DB - RC.DE, WE, n1, &bars[islot]);
    } else if (lane < 6) {
      if (hasB) bulk_row(st + 3 * WE + c3 * WB, my_b + (int64_t)gj * n1, ii0 - RC.DB, WB, n1, &bars[islot]);
    }
    ++inflight;
    if (++islot == NS) islot = 0;
    if (++iq == iRr + 2) {
      iq = 0;
      ii += tw;
      if (ii < ms.nitems) item_geom(ii, ii0, ir0, iRr);
    }
  };
  int wslot = 0;
  unsigned wpar = 0u;
  // wait for the next stage (all lanes agree); on a timeout drain what is in flight
  auto ready = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[wslot], (wpar >> wslot) & 1u, limit_ns));
    if (!ok) {
      if (lane == 0) atomicOr(err, ERRBIT_TIMEOUT);
      int sl = wslot;
      unsigned par = wpar;
      for (int m = 0; m < inflight; ++m) {
        mbar_wait(&bars[sl], (par >> sl) & 1u, limit_ns);
        par ^= 1u << sl;
        if (++sl == NS) sl = 0;
      }
      return false;
    }
    wpar ^= 1u << wslot;
    if (++wslot == NS) wslot = 0;
    --inflight;
    return true;
  };

  for (int k = 0; k < NS; ++k) issue();
  for (int it = gw; it < ms.nitems; it += tw) {
    int i0, r0, Rr;
    item_geom(it, i0, r0, Rr);
    int cslot = wslot;  // slot of stage q
    if (!ready()) return;
    for (int q = 0; q <= Rr; ++q) {
      const int nslot = wslot;  // slot of stage q+1
      const int t = r0 - 1 + q;
      // J row t (Ampere of rows q >= 1): the lane's first column groups loaded
      // before the row's Faraday, which covers the latency
      T jr[kMarchJGroups][3][V];
      const int64_t jrow = (int64_t)(q >= 1 ? t : 0) * n1 + i0;
      const T* jg[3] = {f.j[0] + jrow, f.j[1] + jrow, f.j[2] + jrow};
      if (q >= 1) {
        const int nA = min(SW, n1 - i0);
#pragma unroll
        for (int m = 0; m < kMarchJGroups; ++m) {
          const int oc = (lane + 32 * m) * V;
          if (oc < nA) {
            vld_global<true>(jr[m][0], jg[0] + oc);
            vld_global<true>(jr[m][1], jg[1] + oc);
            vld_global<true>(jr[m][2], jg[2] + oc);
          }
        }
      }
      if (!ready()) return;
      const T* sq = wbase + cslot * ms.stage_elems;   // rows t
      const T* sq1 = wbase + nslot * ms.stage_elems;  // E row t+1
      T* bn = bnew + (q & 1) * 3 * WB;
      march_faraday<T, MT>(sq, sq1, bn, WE, WB, s, lane);
      __syncwarp();
      if (q >= 1)
        march_ampere_jr<T, MT, kMarchJGroups>(sq, bn, bnew + ((q - 1) & 1) * 3 * WB, t, i0, n1, WE,
                                              WB, SW, s, dt, o.e, o.b, jr, jg, lane);
      // stage q is consumed: its slot takes the next stage in the stream
      fence_proxy_async();
      __syncwarp();
      issue();
      cslot = nslot;
    }
    issue();  // the slot of the item's last E row
  }
}


// 3D rows streamed per warp.  Work item = (strip of SW x1 columns, x3 plane k,
// chunk of R x2 rows), k varying fastest over consecutive items so that the
// warps reading the neighbouring planes run at the same time (their common
// rows then come from L2).  Stage q holds the rows t = r0-1+q of E^n at planes
// k-1, k, k+1, of B^{n-1/2} at k-1, k and of J at k (field_rows.cuh,
// march_row3); the plane k-1 B1, B2 of Ampere's x3 difference are recomputed
// per item instead of being exchanged between warps.
template <typename T, int MT>
__global__ void __launch_bounds__(512, 1) field_march3_kernel(FieldPtrs<T> f, OutPtrs<T> o,
                                                           GridArgs g, StencilArgs<T> s,
                                                           MarchShape ms, unsigned* err) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  extern __shared__ __align__(128) unsigned char smem_m[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2];
  const int SW = ms.SW, NS = ms.NS, WE = ms.WE, WB = ms.WB;
  const T dt = (T)g.dt;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_m) + wib * NS;
  T* wbase = reinterpret_cast<T*>(smem_m + ms.bar_bytes) + (size_t)wib * ms.warp_elems;
  T* bnew = wbase + NS * ms.stage_elems;  // [2 rows][3 components][WB], plane k
  T* bk = bnew + 6 * WB;                  // [2 components][WB], plane k-1, current row
  const long long limit_ns = 2000000000LL;
  if (lane == 0) {
    for (int m = 0; m < NS; ++m) mbar_init(&bars[m]);
    mbar_init_fence();
  }
  __syncwarp();
  const int gw = blockIdx.x * nw + wib, tw = gridDim.x * nw;
  int ii = gw, iq = 0, islot = 0, inflight = 0;
  int ii0 = 0, ik = 0, ir0 = 0, iRr = 0;
  auto item_geom = [&](int it, int& i0, int& k, int& r0, int& Rr) {
    const int strip = it % ms.nstrips;
    const int rest = it / ms.nstrips;
    k = rest % n3;
    r0 = (rest / n3) * ms.R;
    i0 = strip * SW;
    Rr = min(ms.R, n2 - r0);
  };
  if (ii < ms.nitems) item_geom(ii, ii0, ik, ir0, iRr);
  const int64_t plane = (int64_t)n1 * n2;
  auto issue = [&]() {
    if (ii >= ms.nitems) return;
    T* st = wbase + islot * ms.stage_elems;
    const int t = ir0 - 1 + iq;
    const int gj = t < 0 ? t + n2 : (t >= n2 ? t - n2 : t);
    const bool hasB = iq <= iRr, hasJ = iq >= 1 && iq <= iRr;
    const int SWr = min(SW, n1 - ii0);
    if (lane == 0)
      mbar_expect_tx(&bars[islot], (uint32_t)((9 * WE + (hasB ? 6 * WB : 0) + (hasJ ? 3 * SWr : 0)) *
                                              sizeof(T)));
    __syncwarp();
    if (lane < 9) {          // E: component lane % 3 at plane k - 1 + lane / 3
      const int c = lane % 3, p = lane / 3;
      const int gk = pwrap(ik - 1 + p, n3);
      bulk_row(st + lane * WE, f.e[c] + gk * plane + (int64_t)gj * n1, ii0 - RC.DB - RC.DE, WE, n1,
               &bars[islot]);
    } else if (lane < 15) {  // B: planes k - 1, k
      const int l = lane - 9, c = l % 3, p = l / 3;
      const int gk = pwrap(ik - 1 + p, n3);
      if (hasB)
        bulk_row(st + 9 * WE + l * WB, f.b[c] + gk * plane + (int64_t)gj * n1, ii0 - RC.DB, WB, n1,
                 &bars[islot]);
    } else if (lane < 18) {  // J: plane k, row t of the item
      const int c = lane - 15;
      if (hasJ)
        bulk_g2s(st + 9 * WE + 6 * WB + c * SW, f.j[c] + ik * plane + (int64_t)t * n1 + ii0,
                 (uint32_t)(SWr * sizeof(T)), &bars[islot]);
    }
    ++inflight;
    if (++islot == NS) islot = 0;
    if (++iq == iRr + 2) {
      iq = 0;
      ii += tw;
      if (ii < ms.nitems) item_geom(ii, ii0, ik, ir0, iRr);
    }
  };
  int wslot = 0;
  unsigned wpar = 0u;
  auto ready = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[wslot], (wpar >> wslot) & 1u, limit_ns));
    if (!ok) {
      if (lane == 0) atomicOr(err, ERRBIT_TIMEOUT);
      int sl = wslot;
      unsigned par = wpar;
      for (int m = 0; m < inflight; ++m) {
        mbar_wait(&bars[sl], (par >> sl) & 1u, limit_ns);
        par ^= 1u << sl;
        if (++sl == NS) sl = 0;
      }
      return false;
    }
    wpar ^= 1u << wslot;
    if (++wslot == NS) wslot = 0;
    --inflight;
    return true;
  };

  for (int m = 0; m < NS; ++m) issue();
  for (int it = gw; it < ms.nitems; it += tw) {
    int i0, k, r0, Rr;
    item_geom(it, i0, k, r0, Rr);
    int cslot = wslot;
    if (!ready()) return;
    for (int q = 0; q <= Rr; ++q) {
      const int nslot = wslot;
      if (!ready()) return;
      const T* sq = wbase + cslot * ms.stage_elems;
      const T* sq1 = wbase + nslot * ms.stage_elems;
      march_row3<T, MT>(sq, sq1, bnew, bk, q, r0 - 1 + q, k, i0, n1, n2, WE, WB, SW, s, dt, o.e,
                        o.b, lane);
      fence_proxy_async();
      __syncwarp();
      issue();
      cslot = nslot;
    }
    issue();
  }
}

// 3D rows streamed along x2 by a CTA of P warps over a group of P consecutive
// x3 planes, warp w on plane k0+w.  Work item = (strip of SW x1 columns, plane
// group, chunk of R x2 rows), the strip varying fastest.  Stage q holds the
// rows t = r0-1+q of E^n at planes k0-1 .. k0+P and of B^{n-1/2} at k0-1 ..
// k0+P-1 (march_layout.cuh, Planes3), staged once for the group by up to 6P+7 bulk
// copies, spread over the warps, on one mbarrier; J is read from global memory
// into registers at the start of the row.  Per row:
// Faraday (planes3_faraday), a CTA barrier (the x3 difference of plane k reads
// the Faraday result of plane k-1), Ampere (planes3_ampere), a CTA barrier
// after which the consumed stage's slot takes the next stage of the stream.
// A staging wait that runs out is agreed on by every warp at the first barrier
// after it: the CTA then waits (bounded) for its copies in flight and returns.
template <typename T, int MT>
__global__ void __launch_bounds__(256, 2) field_planes3_kernel(FieldPtrs<T> f, OutPtrs<T> o,
                                                            GridArgs g, StencilArgs<T> s,
                                                            MarchShape ms, unsigned* err) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  extern __shared__ __align__(128) unsigned char smem_m[];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, P = blockDim.x >> 5;
  const int n1 = g.n[0], n2 = g.n[1], n3 = g.n[2];
  const int SW = ms.SW, NS = ms.NS, WE = ms.WE, WB = ms.WB;
  const Planes3 L{P, WE, WB, SW};
  const T dt = (T)g.dt;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_m);
  T* sbase = reinterpret_cast<T*>(smem_m + ms.bar_bytes);
  // per warp: B^{n+1/2} row t of its plane [3][WB], then B1 B3 of row t-1 over the
  // strip [2][SW]; then B1 B2 of plane k0-1, row t [2][WB]
  T* bnew = sbase + (size_t)NS * ms.stage_elems;
  T* bn = bnew + (size_t)w * L.warp_elems();
  T* bm = bn + 3 * WB;
  T* brec = bnew + (size_t)P * L.warp_elems();
  const long long limit_ns = 2000000000LL;
  if (tid == 0) {
    for (int m = 0; m < NS; ++m) mbar_init(&bars[m]);
    mbar_init_fence();
  }
  __syncthreads();
  const int ngroups = (n3 + P - 1) / P;
  const int64_t plane = (int64_t)n1 * n2;
  auto item_geom = [&](int it, int& i0, int& k0, int& Pg, int& r0, int& Rr) {
    const int strip = it % ms.nstrips;
    const int rest = it / ms.nstrips;
    k0 = (rest % ngroups) * P;
    Pg = min(P, n3 - k0);
    r0 = (rest / ngroups) * ms.R;
    Rr = min(ms.R, n2 - r0);
    i0 = strip * SW;
  };
  // stream cursor, identical in every thread: item ii (geometry cached) and
  // stage iq of the item, filling ring slot islot
  struct Cursor {
    int ii, iq, i0, k0, Pg, r0, Rr;
  };
  auto cur_start = [&](Cursor& c, int it) {
    c.ii = it;
    c.iq = 0;
    if (it < ms.nitems) item_geom(it, c.i0, c.k0, c.Pg, c.r0, c.Rr);
  };
  auto cur_next = [&](Cursor& c) {
    if (c.ii >= ms.nitems) return;
    if (++c.iq == c.Rr + 2) cur_start(c, c.ii + gridDim.x);
  };
  // copies of a stage: E rows, B rows (stages 0 .. Rr)
  auto counts = [&](const Cursor& c, int& nEc, int& nBc) {
    nEc = 3 * (c.Pg + 1) + 2;
    nBc = c.iq <= c.Rr ? 2 + 3 * c.Pg : 0;
  };
  // this thread's copy of the stage (copy ci = lane P + w, spread over the
  // warps): W values of the periodic grid row `src` from column c0 into offset
  // dst of the stage; false if the thread has none
  const int ci = lane * P + w;
  auto my_copy = [&](const Cursor& c, int& dst, const T*& src, int& c0, int& W) {
    int nEc, nBc;
    counts(c, nEc, nBc);
    const int t = c.r0 - 1 + c.iq;
    const int gj = t < 0 ? t + n2 : (t >= n2 ? t - n2 : t);
    if (ci < nEc) {  // E: plane k0-1+pe, component cc
      const int pe = ci / 3, cc = ci - 3 * pe;
      dst = L.er(pe, cc);
      src = f.e[cc] + pwrap(c.k0 - 1 + pe, n3) * plane + (int64_t)gj * n1;
      c0 = c.i0 - RC.DB - RC.DE;
      W = WE;
    } else if (ci < nEc + nBc) {  // B: B1 B2 of plane k0-1, then B1 B2 B3 of the planes
      const int cb = ci - nEc;
      const int pb = cb < 2 ? 0 : 1 + (cb - 2) / 3;
      const int cc = cb < 2 ? cb : (cb - 2) - 3 * (pb - 1);
      dst = L.br(pb, cc);
      src = f.b[cc] + pwrap(c.k0 - 1 + pb, n3) * plane + (int64_t)gj * n1;
      c0 = c.i0 - RC.DB;
      W = WB;
    } else {
      return false;
    }
    return true;
  };
  Cursor ic;
  cur_start(ic, blockIdx.x);
  int islot = 0, inflight = 0;
  auto arm = [&]() {
    if (ic.ii >= ms.nitems || tid != 0) return;
    int nEc, nBc;
    counts(ic, nEc, nBc);
    mbar_expect_tx(&bars[islot], (uint32_t)(((int64_t)nEc * WE + (int64_t)nBc * WB) * sizeof(T)));
  };
  auto copies = [&]() {
    if (ic.ii >= ms.nitems) return;
    int dst, c0, W;
    const T* src;
    T* st = sbase + (size_t)islot * ms.stage_elems;
    if (my_copy(ic, dst, src, c0, W)) bulk_row(st + dst, src, c0, W, n1, &bars[islot]);
    ++inflight;
    if (++islot == NS) islot = 0;
    cur_next(ic);
  };
  // waits are taken in issue order: wslot is the next slot to wait on, bit m
  // of wpar the parity its barrier completes next
  int wslot = 0;
  unsigned wpar = 0u;
  auto ready = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[wslot], (wpar >> wslot) & 1u, limit_ns));
    if (!ok) {
      if (lane == 0) atomicOr(err, ERRBIT_TIMEOUT);
      return false;
    }
    wpar ^= 1u << wslot;
    if (++wslot == NS) wslot = 0;
    --inflight;
    return true;
  };
  auto drain = [&]() {
    int sl = wslot;
    unsigned par = wpar;
    for (int m = 0; m < inflight; ++m) {
      mbar_wait(&bars[sl], (par >> sl) & 1u, limit_ns);
      par ^= 1u << sl;
      if (++sl == NS) sl = 0;
    }
  };

  for (int m = 0; m < NS; ++m) {
    arm();
    __syncthreads();
    copies();
  }
  for (int it = blockIdx.x; it < ms.nitems; it += gridDim.x) {
    int i0, k0, Pg, r0, Rr;
    item_geom(it, i0, k0, Pg, r0, Rr);
    int cslot = wslot;
    bool ok = ready();
    for (int q = 0; q <= Rr; ++q) {
      const int nslot = wslot;
      const int t = r0 - 1 + q;
      // J row t of the warp's plane for Ampere, the lane's first column group
      // loaded before Faraday so that Faraday covers the latency
      const bool amp = q >= 1 && w < Pg;
      T j0[3][V];
      const T* jt[3] = {nullptr, nullptr, nullptr};
      if (amp) {
        const int64_t jrow = ((int64_t)(k0 + w) * n2 + t) * n1 + i0;
        jt[0] = f.j[0] + jrow;
        jt[1] = f.j[1] + jrow;
        jt[2] = f.j[2] + jrow;
        if (lane * V < min(SW, n1 - i0)) {
          vld_global<true>(j0[0], jt[0] + lane * V);
          vld_global<true>(j0[1], jt[1] + lane * V);
          vld_global<true>(j0[2], jt[2] + lane * V);
        }
      }
      ok = ok && ready();
      const T* sq = sbase + (size_t)cslot * ms.stage_elems;   // rows t
      const T* sq1 = sbase + (size_t)nslot * ms.stage_elems;  // E rows t+1
      if (w < Pg) planes3_faraday<T, MT>(sq, sq1, bn, brec, w, Pg, L, s, lane);
      if (q == 0 && w < Pg) {
        // B1, B3 of row r0-1 over the strip, for the x2 differences of row r0
        __syncwarp();
        for (int gq = lane; gq < SW / V; gq += 32) {
          T b[V];
          vld(b, bn + RC.DB + gq * V);
          vst(bm + gq * V, b);
          vld(b, bn + 2 * WB + RC.DB + gq * V);
          vst(bm + SW + gq * V, b);
        }
      }
      if (__syncthreads_or(!ok)) {
        drain();
        return;
      }
      if (amp) {
        const T* bk = w == 0 ? brec : bnew + (size_t)(w - 1) * L.warp_elems();
        planes3_ampere<T, MT>(sq, bn, bm, bk, jt, j0, w, t, k0 + w, i0, n1, n2, L, s, dt, o.e, o.b,
                              lane);
      }
      // stage q is consumed by every warp: its slot takes the next stage
      fence_proxy_async();
      arm();
      __syncthreads();
      copies();
      cslot = nslot;
    }
    arm();  // the slot of the item's last E row
    __syncthreads();
    copies();
  }
}

// Time-centred B^n = B^{n-1/2} - (dt/2) d_E x E^n at every cell, for read-out.
template <typename T, int NDIM>
__global__ void bbar_kernel(FieldPtrs<T> f, GridArgs g, StencilArgs<T> s, double* out,
                            int comp) {
  const int n1 = g.n[0], n2 = g.n[1], n3 = (NDIM == 3) ? g.n[2] : 1;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(q % n1);
    int64_t r = q / n1;
    int j = (int)(r % n2), k = (int)(r / n2);
    auto at = [&](const T* a, int di, int dj, int dk) -> double {
      return (double)a[((int64_t)wrap_index(k + dk, n3) * n2 + wrap_index(j + dj, n2)) * n1 +
                       wrap_index(i + di, n1)];
    };
    double curl = 0.0;
    auto dE1 = [&](const T* a) {
      double acc = 0.0;
      for (int m = 1; m <= s.M; ++m) acc += (double)s.kE[m - 1] * (at(a, m, 0, 0) - at(a, 1 - m, 0, 0));
      return acc;
    };
    if (comp == 0)
      curl = (double)s.y2 * (at(f.e[2], 0, 1, 0) - at(f.e[2], 0, 0, 0)) -
             (NDIM == 3 ? (double)s.y3 * (at(f.e[1], 0, 0, 1) - at(f.e[1], 0, 0, 0)) : 0.0);
    else if (comp == 1)
      curl = (NDIM == 3 ? (double)s.y3 * (at(f.e[0], 0, 0, 1) - at(f.e[0], 0, 0, 0)) : 0.0) -
             dE1(f.e[2]);
    else
      curl = dE1(f.e[1]) - (double)s.y2 * (at(f.e[0], 0, 1, 0) - at(f.e[0], 0, 0, 0));
    out[q] = (double)f.b[comp][q] - 0.5 * curl;
  }
}

// x1 current correction (Sec. 3.3): J1 <- P^{-1} J1 per x1 row, applied as the
// circular convolution with the taps g_m of the exact inverse of the circulant P
// (symbol [k]_Yee/[k]_B1): J1'_i = sum_{m<count} g_{lo+m} J1_{i+lo+m} (periodic
// in i), taps[m] = g_{lo+m}, stored in the field precision T and accumulated in
// T.  Every form below adds the products in ascending m with one fused
// multiply-add each, so all three give bit-identical results.
//
// Rows form (in place): a CTA stages one whole x1 row, with `count - 1` wrapped
// values past its end, in shared memory, then overwrites the row.  Thread t
// forms the V = 16/sizeof(T) consecutive outputs V*q (q = t, t + 256, ...) from
// a sliding register window: per V taps one 16-byte shared load of inputs, one
// (broadcast) of taps, V*V products.
constexpr int kCorrT = 256, kCorrR = 4, kCorrW = kCorrT * kCorrR;

inline size_t correct_j1_rows_smem(int n1, int count, size_t tsize) {
  const int V = (int)(16 / tsize);
  const int cpad = ceil_to(count, V);
  return (size_t)(2 * cpad + ceil_to(n1, V)) * tsize;
}

inline size_t correct_j1_smem(int count, size_t tsize) {
  return (size_t)(kCorrW + 2 * count) * tsize;
}

template <typename T>
__global__ void __launch_bounds__(kCorrT) correct_j1_rows_kernel(T* __restrict__ j1, GridArgs g,
                                                                 const T* __restrict__ taps,
                                                                 int lo, int count) {
  constexpr int V = VecOf<T>::V;
  extern __shared__ __align__(16) unsigned char corr_smem[];
  const int n1 = g.n[0];
  const int cpad = ceil_to(count, V);
  const int nq = (n1 + V - 1) / V;
  const int span = nq * V + cpad;  // furthest input read: V*(nq-1) + cpad + V - 1
  T* st = reinterpret_cast<T*>(corr_smem);  // cpad taps, zero past count
  T* sx = st + cpad;                        // span staged inputs, 16-byte aligned
  const int tid = threadIdx.x;
  for (int m = tid; m < cpad; m += kCorrT) st[m] = m < count ? taps[m] : (T)0;
  const int64_t rows = g.ncell / n1;
  const bool vec_out = (n1 % V) == 0;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    T* rp = j1 + row * n1;
    __syncthreads();  // the previous row's reads of sx are done
    int w = wrap_index(lo + tid, n1);
    for (int t = tid; t < span; t += kCorrT) {
      sx[t] = rp[w];
      w += kCorrT;
      while (w >= n1) w -= n1;
    }
    __syncthreads();  // every read of this row precedes the first write
    for (int q = tid; q < nq; q += kCorrT) {
      const T* xb = sx + V * q;
      T win[2 * V], gv[V], acc[V];
#pragma unroll
      for (int j = 0; j < V; ++j) acc[j] = (T)0;
      vld(win, xb);
      for (int k = 0; k < cpad; k += V) {
        vld(win + V, xb + k + V);
        vld(gv, st + k);
#pragma unroll
        for (int s = 0; s < V; ++s)
#pragma unroll
          for (int j = 0; j < V; ++j) acc[j] = fma(gv[s], win[j + s], acc[j]);
#pragma unroll
        for (int j = 0; j < V; ++j) win[j] = win[V + j];
      }
      const int i = V * q;
      if (vec_out) {
        vst(rp + i, acc);
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j)
          if (i + j < n1) rp[i + j] = acc[j];
      }
    }
  }
}

// Segments form (out of place, any row length): a work item is kCorrW outputs of
// one row; the CTA stages in[i0+lo .. i0+lo+kCorrW+count-2] (wrapped) and the
// taps, thread t forms outputs i0 + t + kCorrT*r, r < kCorrR.
template <typename T>
__global__ void __launch_bounds__(kCorrT) correct_j1_kernel(const T* __restrict__ in,
                                                            T* __restrict__ out, GridArgs g,
                                                            const T* __restrict__ taps, int lo,
                                                            int count) {
  extern __shared__ __align__(16) unsigned char corr_smem[];
  T* st = reinterpret_cast<T*>(corr_smem);
  T* sx = st + count;
  const int n1 = g.n[0];
  const int tid = threadIdx.x;
  for (int m = tid; m < count; m += kCorrT) st[m] = taps[m];
  const int segs = (n1 + kCorrW - 1) / kCorrW;
  const int64_t rows = g.ncell / n1;
  const int span = kCorrW + count - 1;
  for (int64_t item = blockIdx.x; item < rows * segs; item += gridDim.x) {
    const int64_t row = item / segs;
    const int i0 = (int)(item - row * segs) * kCorrW;
    const T* rp = in + row * n1;
    __syncthreads();  // the previous item's reads of sx are done
    int w = wrap_index(i0 + lo + tid, n1);
    for (int t = tid; t < span; t += kCorrT) {
      sx[t] = rp[w];
      w += kCorrT;
      while (w >= n1) w -= n1;
    }
    __syncthreads();
    T acc[kCorrR];
#pragma unroll
    for (int r = 0; r < kCorrR; ++r) acc[r] = (T)0;
    const T* xs = sx + tid;
#pragma unroll 4
    for (int m = 0; m < count; ++m) {
      const T gm = st[m];
#pragma unroll
      for (int r = 0; r < kCorrR; ++r) acc[r] = fma(gm, xs[m + kCorrT * r], acc[r]);
    }
    T* op = out + row * n1;
#pragma unroll
    for (int r = 0; r < kCorrR; ++r) {
      const int i = i0 + tid + kCorrT * r;
      if (i < n1) op[i] = acc[r];
    }
  }
}

// Rows too long for the shared-memory form (a non-decaying tap set on a very long
// x1 axis): the same sum, read straight from global memory.
template <typename T>
__global__ void correct_j1_global_kernel(const T* __restrict__ in, T* __restrict__ out,
                                         GridArgs g, const T* __restrict__ taps, int lo,
                                         int count) {
  const int n1 = g.n[0];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const T* rp = in + (q - i);
    T acc = (T)0;
    int w = wrap_index(i + lo, n1);
    for (int m = 0; m < count; ++m) {
      acc = fma(taps[m], rp[w], acc);
      if (++w == n1) w = 0;
    }
    out[q] = acc;
  }
}

template <typename T>
__global__ void convert_in_kernel(T* dst, const double* src, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = (T)src[q];
}

template <typename T>
__global__ void convert_out_kernel(double* dst, const T* src, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = (double)src[q];
}

template <typename T>
__global__ void laser_expand_kernel(FieldPtrs<T> f, GridArgs g, const double* ep,
                                    const double* bp, double w0, double x2c, double x3c) {
  const int n1 = g.n[0], n2 = g.n[1];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const int64_t r = q / n1;
    const int j = (int)(r % n2), k = (int)(r / n2);
    double tr = 1.0;
    if (w0 > 0.0) {
      // E2 and B3 share x2 = (j+1/2) dx2 and x3 = k dx3
      const double d2 = ((j + 0.5) * g.dx[1] - x2c) / w0;
      tr = exp(-d2 * d2);
      if (g.ndim == 3) {
        const double d3 = (k * g.dx[2] - x3c) / w0;
        tr *= exp(-d3 * d3);
      }
    }
    for (int c = 0; c < 3; ++c) {
      f.e[c][q] = (T)0;
      f.b[c][q] = (T)0;
    }
    f.e[1][q] = (T)(ep[i] * tr);
    f.b[2][q] = (T)(bp[i] * tr);
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

template <typename T, int NDIM, int MT>
cudaError_t launch_field_step_mt(const FieldPtrs<T>& f, const OutPtrs<T>& o, const GridArgs& g,
                                 const StencilArgs<T>& s, const FieldTile& tile, unsigned* err,
                                 cudaStream_t st) {
  constexpr int V = VecOf<T>::V;
  const int TX = tile.t[0], TY = tile.t[1], TZ = (NDIM == 3) ? tile.t[2] : 1;
  const int NT = tile.threads > 0 ? tile.threads : 256;
  if (TX % V != 0 || NT % 32 != 0 || NT > 512) return cudaErrorInvalidValue;
  const int M = s.M;
  const int64_t ntiles = (int64_t)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY) *
                         (NDIM == 3 ? (g.n[2] + TZ - 1) / TZ : 1);
  // bulk copies need 16-byte aligned row starts: n1 a multiple of V, aligned arrays
  uintptr_t am = 0;
  for (int c = 0; c < 3; ++c)
    am |= (uintptr_t)f.e[c] | (uintptr_t)f.b[c] | (uintptr_t)f.j[c];
  const bool async_ok = tile.staging != 1 && g.n[0] % V == 0 && (am & 15u) == 0;
  const bool rows_ok = async_ok && tile.staging == 0;   // rows streamed per warp
  cudaError_t e;
  int dev = 0, smem_max = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
      cudaSuccess)
    return e;
  if (NDIM == 2 && rows_ok) {
    // rows streamed per warp: tile = TX x1 columns x TY rows of one warp
    constexpr Reach RC(MT, V);
    MarchShape ms;
    ms.SW = tile.sw;
    ms.R = tile.rows;
    ms.NS = tile.stages;
    const int nw = tile.warps;
    if (ms.SW % V != 0 || ms.SW < V || ms.R < 0 || ms.NS < 2 || ms.NS > 8 || nw < 1 || nw > 16)
      return cudaErrorInvalidValue;
    ms.WE = RC.WE(ms.SW, V);
    ms.WB = RC.WB(ms.SW, V);
    ms.nstrips = (g.n[0] + ms.SW - 1) / ms.SW;
    ms.stage_elems = 3 * (ms.WE + ms.WB);  // J is read from global memory
    ms.warp_elems = ms.NS * ms.stage_elems + 6 * ms.WB;
    ms.bar_bytes = (nw * ms.NS * 8 + 127) / 128 * 128;
    const size_t smem = ms.bar_bytes + (size_t)nw * ms.warp_elems * sizeof(T);
    if (ms.WE <= g.n[0] && smem <= (size_t)smem_max) {
      auto kern = field_march_kernel<T, MT>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int nsm = 0, per_sm = 0;
      if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * nw, smem)) !=
          cudaSuccess)
        return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      if (ms.R == 0) {
        // rows per item so that the items fill the resident warps in one round
        const int64_t tw = (int64_t)nsm * per_sm * nw;
        const int64_t chunks = std::max<int64_t>(1, tw / ms.nstrips);
        ms.R = (int)((g.n[1] + chunks - 1) / chunks);
      }
      ms.nitems = (int)(ms.nstrips * (int64_t)((g.n[1] + ms.R - 1) / ms.R));
      const int64_t grid = std::min<int64_t>((ms.nitems + nw - 1) / nw, (int64_t)nsm * per_sm);
      kern<<<(unsigned)grid, 32 * nw, smem, st>>>(f, o, g, s, ms, err);
      return cudaGetLastError();
    }
  }
  if (NDIM == 3 && rows_ok && tile.warps > 1) {
    // rows streamed along x2 by a CTA of P warps over P consecutive x3 planes
    constexpr Reach RC(MT, V);
    MarchShape ms;
    ms.SW = tile.sw;
    ms.R = tile.rows;
    ms.NS = tile.stages;
    const int P = tile.warps;
    if (ms.SW % V != 0 || ms.SW < V || ms.R < 0 || ms.NS < 2 || ms.NS > 8 || P > 8)
      return cudaErrorInvalidValue;
    ms.WE = RC.WE(ms.SW, V);
    ms.WB = RC.WB(ms.SW, V);
    ms.nstrips = (g.n[0] + ms.SW - 1) / ms.SW;
    ms.stage_elems = (int)planes3_stage_elems(P, ms.SW, ms.WE, ms.WB);
    ms.warp_elems = (int)planes3_cta_elems(P, ms.SW, ms.WE, ms.WB, ms.NS);
    ms.bar_bytes = (ms.NS * 8 + 127) / 128 * 128;
    const size_t smem = ms.bar_bytes + (size_t)ms.warp_elems * sizeof(T);
    if (ms.WE <= g.n[0] && g.n[2] >= 2 && smem <= (size_t)smem_max) {
      auto kern = field_planes3_kernel<T, MT>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int nsm = 0, per_sm = 0;
      if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * P, smem)) !=
          cudaSuccess)
        return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      const int64_t slots = (int64_t)nsm * per_sm;
      const int64_t cols = (int64_t)ms.nstrips * ((g.n[2] + P - 1) / P);
      if (ms.R == 0) ms.R = balanced_rows(g.n[1], cols, slots);
      ms.nitems = (int)(cols * (int64_t)((g.n[1] + ms.R - 1) / ms.R));
      const int64_t grid = std::min<int64_t>(ms.nitems, slots);
      kern<<<(unsigned)grid, 32 * P, smem, st>>>(f, o, g, s, ms, err);
      return cudaGetLastError();
    }
  }
  if (NDIM == 3 && rows_ok) {
    // rows streamed per warp along x2, one x3 plane per item
    constexpr Reach RC(MT, V);
    MarchShape ms;
    ms.SW = tile.sw;
    ms.R = tile.rows;
    ms.NS = tile.stages;
    const int nw = tile.warps;
    if (ms.SW % V != 0 || ms.SW < V || ms.R < 0 || ms.NS < 2 || ms.NS > 8 || nw < 1 || nw > 16)
      return cudaErrorInvalidValue;
    ms.WE = RC.WE(ms.SW, V);
    ms.WB = RC.WB(ms.SW, V);
    ms.nstrips = (g.n[0] + ms.SW - 1) / ms.SW;
    ms.stage_elems = 9 * ms.WE + 6 * ms.WB + 3 * ms.SW;
    ms.warp_elems = ms.NS * ms.stage_elems + 8 * ms.WB;
    ms.bar_bytes = (nw * ms.NS * 8 + 127) / 128 * 128;
    const size_t smem = ms.bar_bytes + (size_t)nw * ms.warp_elems * sizeof(T);
    if (ms.WE <= g.n[0] && g.n[2] >= 2 && smem <= (size_t)smem_max) {
      auto kern = field_march3_kernel<T, MT>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int nsm = 0, per_sm = 0;
      if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * nw, smem)) !=
          cudaSuccess)
        return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      const int64_t tw = (int64_t)nsm * per_sm * nw;
      const int64_t cols = (int64_t)ms.nstrips * g.n[2];
      if (ms.R == 0) {
        const int64_t chunks = std::max<int64_t>(1, tw / cols);
        ms.R = (int)((g.n[1] + chunks - 1) / chunks);
      }
      ms.nitems = (int)(cols * (int64_t)((g.n[1] + ms.R - 1) / ms.R));
      const int64_t grid = std::min<int64_t>((ms.nitems + nw - 1) / nw, (int64_t)nsm * per_sm);
      kern<<<(unsigned)grid, 32 * nw, smem, st>>>(f, o, g, s, ms, err);
      return cudaGetLastError();
    }
  }
  const size_t tile_elems = field_tile_smem_elems(NDIM, TX, TY, TZ, M, (int)sizeof(T));
  const int buf_elems = (int)(tile_elems + (size_t)3 * TX * TY * TZ);
  const size_t smem_async = 128 + 2 * (size_t)buf_elems * sizeof(T);
  if (async_ok && smem_async <= (size_t)smem_max) {
    const size_t smem = smem_async;
    auto kern = field_step_tma_kernel<T, NDIM, MT>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess)
      return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
    kern<<<(unsigned)grid, NT, smem, st>>>(f, o, g, s, TX, TY, TZ, (int)ntiles, buf_elems, err);
    return cudaGetLastError();
  }
  const size_t smem = tile_elems * sizeof(T);
  e = cudaFuncSetAttribute(field_step_kernel<T, NDIM, MT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  field_step_kernel<T, NDIM, MT><<<(unsigned)ntiles, NT, smem, st>>>(f, o, g, s, TX, TY, TZ);
  return cudaGetLastError();
}

template <typename T, int NDIM>
cudaError_t launch_field_step_nd(const FieldPtrs<T>& f, const OutPtrs<T>& o, const GridArgs& g,
                                 const StencilArgs<T>& s, const FieldTile& tile, unsigned* err,
                                 cudaStream_t st) {
  switch (stencil_mt(s.M)) {
    case 8:
      return launch_field_step_mt<T, NDIM, 8>(f, o, g, s, tile, err, st);
    case 16:
      return launch_field_step_mt<T, NDIM, 16>(f, o, g, s, tile, err, st);
    default:
      return launch_field_step_mt<T, NDIM, 32>(f, o, g, s, tile, err, st);
  }
}

template <typename T>
cudaError_t launch_field_step(const FieldPtrs<T>& f, const FieldPtrs<T>& out, const GridArgs& g,
                              const StencilArgs<T>& s, const FieldTile& tile, unsigned* err,
                              cudaStream_t st) {
  OutPtrs<T> o;
  for (int c = 0; c < 3; ++c) {
    o.e[c] = out.e[c];
    o.b[c] = out.b[c];
  }
  if (g.ndim == 3) return launch_field_step_nd<T, 3>(f, o, g, s, tile, err, st);
  return launch_field_step_nd<T, 2>(f, o, g, s, tile, err, st);
}

template <typename T>
cudaError_t launch_bbar(const FieldPtrs<T>& f, const GridArgs& g, const StencilArgs<T>& s,
                        double* out, int comp, cudaStream_t st) {
  if (g.ndim == 3)
    bbar_kernel<T, 3><<<grid_for(g.ncell), 256, 0, st>>>(f, g, s, out, comp);
  else
    bbar_kernel<T, 2><<<grid_for(g.ncell), 256, 0, st>>>(f, g, s, out, comp);
  return cudaGetLastError();
}

// CTAs of `threads` threads and `smem` bytes each that fit one SM at once
inline int ctas_per_sm(size_t smem, int threads) {
  const int by_smem = (int)((228 * 1024) / (smem + 1024));
  return std::max(1, std::min(2048 / threads, by_smem));
}

template <typename T>
cudaError_t launch_correct_j1(T* j1, T* tmp, const GridArgs& g, const T* taps, int lo, int count,
                              int path, cudaStream_t st) {
  constexpr size_t kMaxSmem = 200 * 1024;
  const int64_t rows = g.ncell / g.n[0];
  size_t smem = correct_j1_rows_smem(g.n[0], count, sizeof(T));
  if (path == 0) path = smem <= kMaxSmem ? 1 : correct_j1_smem(count, sizeof(T)) <= kMaxSmem ? 2 : 3;
  if (path == 1) {
    if (smem > kMaxSmem) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(correct_j1_rows_kernel<T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    const int grid = (int)std::min<int64_t>(rows, 152 * ctas_per_sm(smem, kCorrT));
    correct_j1_rows_kernel<T><<<grid, kCorrT, smem, st>>>(j1, g, taps, lo, count);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemcpyAsync(tmp, j1, sizeof(T) * g.ncell, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  if (path == 2) {
    smem = correct_j1_smem(count, sizeof(T));
    if (smem > kMaxSmem) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(correct_j1_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
    }
    const int64_t items = rows * ((g.n[0] + kCorrW - 1) / kCorrW);
    const int grid = (int)std::min<int64_t>(items, 152 * ctas_per_sm(smem, kCorrT));
    correct_j1_kernel<T><<<grid, kCorrT, smem, st>>>(tmp, j1, g, taps, lo, count);
  } else {
    correct_j1_global_kernel<T><<<grid_for(g.ncell), 256, 0, st>>>(tmp, j1, g, taps, lo, count);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_in(T* dst, const double* src, int64_t n, cudaStream_t st) {
  convert_in_kernel<T><<<grid_for(n), 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert_out(double* dst, const T* src, int64_t n, cudaStream_t st) {
  convert_out_kernel<T><<<grid_for(n), 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_laser_expand(const FieldPtrs<T>& f, const GridArgs& g, const double* eprof,
                                const double* bprof, double w0, double x2c, double x3c,
                                cudaStream_t st) {
  laser_expand_kernel<T><<<grid_for(g.ncell), 256, 0, st>>>(f, g, eprof, bprof, w0, x2c, x3c);
  return cudaGetLastError();
}

#define PIC_INST(T)                                                                          \
  template cudaError_t launch_field_step<T>(const FieldPtrs<T>&, const FieldPtrs<T>&,       \
                                            const GridArgs&, const StencilArgs<T>&,         \
                                            const FieldTile&, unsigned*, cudaStream_t);     \
  template cudaError_t launch_bbar<T>(const FieldPtrs<T>&, const GridArgs&,                 \
                                      const StencilArgs<T>&, double*, int, cudaStream_t);   \
  template cudaError_t launch_correct_j1<T>(T*, T*, const GridArgs&, const T*, int, int, int,\
                                            cudaStream_t);                                  \
  template cudaError_t launch_convert_in<T>(T*, const double*, int64_t, cudaStream_t);      \
  template cudaError_t launch_convert_out<T>(double*, const T*, int64_t, cudaStream_t);     \
  template cudaError_t launch_laser_expand<T>(const FieldPtrs<T>&, const GridArgs&,         \
                                              const double*, const double*, double, double, \
                                              double, cudaStream_t);
PIC_INST(double)
PIC_INST(float)
PIC_INST(dfl)
#undef PIC_INST

}  // namespace pic
