// batch.cu -- ensembles of independent 2D runs advanced by one persistent kernel.
//
// Every run keeps its own fields (in one pool), particles and step count.  One
// cooperative launch loops over the steps; in each step its warps take work
// items -- row strips of any run's field update (field_rows.cuh: Faraday and
// Ampere streamed along x2 through a per-warp ring of bulk-copied rows), taken
// from a per-step atomic counter, and 32-particle chunks of any run
// (gather/push/move/deposit from global memory, particle_core.cuh) -- and meet
// at a grid barrier before the next step.
// Field buffers alternate between two parities per run, so a step only reads
// what the previous step wrote.  When some particle deposits current, a step
// has two phases (particles, barrier, fields, barrier) and the field tiles clear
// the current they consume.  Every barrier wait is bounded in time: on expiry
// the kernel latches a timeout bit and returns instead of spinning on.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "field_rows.cuh"
#include "field_tile.cuh"
#include "correction_host.h"
#include "laser_host.h"
#include "particle_core.cuh"

using namespace pic;

namespace {

struct RunInfo {
  int n1, n2;
  int ld;           // row pitch in the pool: n1 + 2 gh rounded up to 16 bytes of the field type
  int64_t off;      // first value of the run in each pool array (256-byte aligned)
  int nstrips;      // x1 strips of the run for the current strip width
  int64_t p0, p1;   // particle range
  int64_t nsteps;   // steps of the current pic_batch_run
  int cur;          // parity of the buffers holding the run's state
  int toff, tcount, tlo;  // x1 current-correction taps of the run's row length
};

// Shape of the field work: strips of SW x1 columns by R rows, a ring of NS row
// stages per warp (see field_rows.cuh for the stage layout), NW warps per CTA.
struct StripShape {
  int SW, R, NS, NW;
  int WE, WB, stage_elems, warp_elems, hdr_bytes;
};

template <typename T>
struct BatchArgs {
  RunInfo* runs;
  const int2* items;  // [0, nfield): (run, chunk*nstrips + strip); then (run, particle chunk);
                      // the last ncorr: (run, row) of the x1 current correction
  int nitems, nfield, ncorr;
  const T* taps;      // correction taps of all row lengths (RunInfo::toff)
  unsigned* ctr;      // two per-step counters of taken field items (alternating steps)
  StripShape sh;
  int gh;             // ghost columns on each side of every pool row (the x1 stencils' reach)
  T* pool;            // [parity 0: E1 E2 E3 B1 B2 B3][parity 1: ...][J1 J2 J3], `total` cells each
  int64_t total;
  PartPtrs parts;
  StencilArgs<T> s;
  GridArgs gbase;     // dx, inv_dx, dx_dt, dt (sizes per run)
  PartArgs a;
  int64_t max_steps;
  int has_current;
  unsigned* bar;      // monotonically increasing arrival count
  unsigned* err;
  unsigned expected;  // CTAs each barrier waits for
  long long timeout_ns;
};

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a bounded wait.  Returns false (after latching the timeout
// bit) if the other CTAs did not arrive within A.timeout_ns.
template <typename T>
__device__ bool grid_wait(const BatchArgs<T>& A, unsigned& epoch) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(A.bar, 1u);
    ++epoch;
    const unsigned target = epoch * A.expected;
    const long long t0 = globaltimer_ns();
    for (;;) {
      const unsigned v = *((volatile unsigned*)A.bar);
      if (v >= target) break;
      if (globaltimer_ns() - t0 > A.timeout_ns) {
        atomicOr(A.err, ERRBIT_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ T* pool_ptr(const BatchArgs<T>& A, int slot, int64_t off) {
  return A.pool + (int64_t)slot * A.total + off;
}

// column 0 of row 0 of a run's array (rows are ld apart, with gh ghost columns
// on each side mirroring the periodic row)
template <typename T>
__device__ __forceinline__ T* run_ptr(const BatchArgs<T>& A, int slot, const RunInfo& R) {
  return pool_ptr(A, slot, R.off) + A.gh;
}

// 32 particles of a run per warp (gather E^n and time-centred B^n from the
// run's fields, push, move, deposit when the particles carry charge)
template <typename T>
__device__ void particle_chunk(const BatchArgs<T>& A, const StencilArgs<T>* sp, const RunInfo& R,
                               int chunk, int par, int lane) {
  const int64_t q = R.p0 + (int64_t)chunk * 32 + lane;
  if (q >= R.p1) return;
  GridArgs g = A.gbase;
  g.n[0] = R.n1;
  g.n[1] = R.n2;
  g.len[0] = R.n1 * g.dx[0];
  g.len[1] = R.n2 * g.dx[1];
  g.ncell = (int64_t)R.n1 * R.n2;
  GlobView<T, true> ve[3];
  BbarView<T, 2, true> vb[3];
  GlobAcc<T> acc[3];
  const T* e[3];
  for (int c = 0; c < 3; ++c) e[c] = run_ptr(A, par * 6 + c, R);
  for (int c = 0; c < 3; ++c) {
    ve[c] = GlobView<T, true>{e[c], R.n1, R.n2, 1, R.ld};
    vb[c] = BbarView<T, 2, true>{{e[0], e[1], e[2]}, run_ptr(A, par * 6 + 3 + c, R), c,
                                 R.n1, R.n2, 1, sp, R.ld};
    acc[c] = GlobAcc<T>{run_ptr(A, 12 + c, R), R.n1, R.n2, 1, R.ld};
  }
  int li[3] = {0, 0, 0};
  T fr[3] = {0, 0, 0};
  for (int d = 0; d < 2; ++d) {
    const double c = A.parts.x[d][q] * g.inv_dx[d];
    double frac;
    li[d] = floor_split(c, frac);
    fr[d] = to_prec<T>(frac);
  }
  advance_particle<T, 2>(ve, vb, acc, A.parts, q, li, fr, li, g, A.a, A.err);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Field item being streamed by a warp
template <typename T>
struct StripItem {
  const T* e[3];
  const T* b[3];
  T* j[3];
  T* eo[3];
  T* bo[3];
  int n1, n2, p1, i0, r0, Rr;
  bool ghosted;  // n1 >= gh: every region row is one contiguous range of a pool row
};

template <typename T, int MT>
__device__ __forceinline__ void strip_item(const BatchArgs<T>& A, int k, int64_t step,
                                           StripItem<T>& it) {
  constexpr int V = VecOf<T>::V;
  const int2 w = A.items[k];
  const RunInfo R = A.runs[w.x];
  const int chunk = w.y / R.nstrips;
  it.n1 = R.n1;
  it.n2 = R.n2;
  it.p1 = R.ld;
  it.i0 = (w.y - chunk * R.nstrips) * A.sh.SW;
  it.r0 = chunk * A.sh.R;
  it.Rr = min(A.sh.R, R.n2 - it.r0);
  const int par = (R.cur + (int)step) & 1;
  for (int c = 0; c < 3; ++c) {
    it.e[c] = run_ptr(A, par * 6 + c, R);
    it.b[c] = run_ptr(A, par * 6 + 3 + c, R);
    it.eo[c] = run_ptr(A, (1 - par) * 6 + c, R);
    it.bo[c] = run_ptr(A, (1 - par) * 6 + 3 + c, R);
    it.j[c] = run_ptr(A, 12 + c, R);
  }
  it.ghosted = R.n1 >= A.gh;
}

// next field item of this step not yet taken by any warp whose run is still
// stepping; -1 when none is left (all lanes get the same answer)
template <typename T>
__device__ __forceinline__ int take_item(const BatchArgs<T>& A, unsigned* ctr, int64_t step,
                                         int lane) {
  for (;;) {
    int k = 0;
    if (lane == 0) k = (int)atomicAdd(ctr, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= A.nfield) return -1;
    const int2 w = A.items[k];
    if (step < A.runs[w.x].nsteps) return k;
  }
}

// x1 current correction of one J1 row of a run (Sec. 3.3, Eq. (23)): the row
// (with count - 1 wrapped values past its end) and the run's taps are staged in
// the warp's shared memory, then the row is overwritten with the periodic
// convolution J1'_i = sum_m g_{lo+m} J1_{i+lo+m}.  Lane l forms the V outputs
// V*q (q = l, l + 32, ...) from a sliding register window, adding the products
// in ascending m with one fused multiply-add each, as the single-grid kernels
// do: the same row and taps give the same bits.
template <typename T>
__device__ void correct_row(const BatchArgs<T>& A, const RunInfo& R, int row, T* ws, int lane) {
  constexpr int V = VecOf<T>::V;
  const int n1 = R.n1, count = R.tcount;
  const int cpad = ceil_to(count, V);
  const int nq = (n1 + V - 1) / V;
  const int span = nq * V + cpad;  // furthest input read: V*(nq-1) + cpad + V - 1
  T* st = ws;
  T* sx = ws + cpad;
  T* rp = run_ptr(A, 12, R) + (int64_t)row * R.ld;
  const T* tp = A.taps + R.toff;
  for (int m = lane; m < cpad; m += 32) st[m] = m < count ? tp[m] : (T)0;
  int w = wrap_index(R.tlo + lane, n1);
  for (int t = lane; t < span; t += 32) {
    sx[t] = rp[w];
    w += 32;
    while (w >= n1) w -= n1;
  }
  __syncwarp();
  for (int q = lane; q < nq; q += 32) {
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
    if (i + V <= n1) {
      vst(rp + i, acc);
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j)
        if (i + j < n1) rp[i + j] = acc[j];
    }
  }
  // the field phase refills this shared memory with bulk copies
  fence_proxy_async();
  __syncwarp();
}

// Ring cursors of a warp (persist across steps; every stage issued in a step is
// consumed in it): next slot to issue into, next slot to wait on, stages in
// flight, and bit k = phase parity slot k's barrier completes next.
struct RingCursor {
  int islot, wslot, inflight;
  unsigned wpar;
};

// The field update of one step for one warp: items are taken from the step's
// counter and their rows streamed through the warp's ring (field_rows.cuh).
// Pool rows carry ghost columns (copies of the periodic row's ends, written by
// the same stores), so each region row is one aligned bulk copy; runs narrower
// than the ghost width fill E and B rows by element-wise cp.async copies
// tracked by the same barriers.  Returns
// false after a staging wait ran out (the copies in flight are drained first).
template <typename T, int MT>
__device__ __forceinline__ bool field_phase(const BatchArgs<T>& A, const StencilArgs<T>& s,
                                            int64_t step, uint64_t* bars, int* slot_item,
                                            T* wbase, RingCursor& rc, int lane) {
  constexpr int V = VecOf<T>::V;
  constexpr Reach RC(MT, V);
  const int SW = A.sh.SW, NS = A.sh.NS, WE = A.sh.WE, WB = A.sh.WB;
  const T dt = (T)A.gbase.dt;
  const bool has_j = A.has_current != 0;
  unsigned* ctr = A.ctr + (step & 1);
  T* bnew = wbase + NS * A.sh.stage_elems;
  const long long limit_ns = 2000000000LL;
  const int c3 = lane % 3;

  // issue cursor: item ik, stage iq
  int ik = take_item<T>(A, ctr, step, lane), iq = 0;
  StripItem<T> is;
  if (ik >= 0) strip_item<T, MT>(A, ik, step, is);
  auto issue = [&]() {
    if (ik < 0) return;
    T* st = wbase + rc.islot * A.sh.stage_elems;
    uint64_t* bar = &bars[rc.islot];
    const int t = is.r0 - 1 + iq;
    const int gj = t < 0 ? t + is.n2 : (t >= is.n2 ? t - is.n2 : t);
    const bool hasB = iq <= is.Rr, hasJ = has_j && iq >= 1 && iq <= is.Rr;
    const int SWr = min(SW, is.n1 - is.i0);
    const int Es = is.i0 - RC.DB - RC.DE, Bs = is.i0 - RC.DB;
    const int SWc = (SWr + V - 1) / V * V;  // J copy width, inside the row pitch
    const int64_t rofs = (int64_t)gj * is.p1;
    if (is.ghosted) {
      // a region row [c0, c0 + W) with c0 >= -gh is contiguous up to column
      // n1 + gh: one bulk copy, cut where the ghost columns end (the columns
      // past that feed no output of the strip inside the run)
      const int WEc = (min(WE, is.n1 + A.gh - Es) + V - 1) / V * V;
      const int WBc = (min(WB, is.n1 + A.gh - Bs) + V - 1) / V * V;
      if (lane == 0) {
        slot_item[rc.islot] = ik;
        mbar_expect_tx(bar, (uint32_t)((3 * WEc + (hasB ? 3 * WBc : 0) + (hasJ ? 3 * SWc : 0)) *
                                       sizeof(T)));
      }
      __syncwarp();
      if (lane < 3) {
        bulk_g2s(st + c3 * WE, is.e[c3] + rofs + Es, (uint32_t)(WEc * sizeof(T)), bar);
      } else if (lane < 6) {
        if (hasB) bulk_g2s(st + 3 * WE + c3 * WB, is.b[c3] + rofs + Bs, (uint32_t)(WBc * sizeof(T)), bar);
      } else if (lane < 9) {
        if (hasJ)
          bulk_g2s(st + 3 * WE + 3 * WB + c3 * SW, is.j[c3] + (int64_t)t * is.p1 + is.i0,
                   (uint32_t)(SWc * sizeof(T)), bar);
      }
    } else {
      // runs narrower than the ghost width: element-wise cp.async with the
      // periodic wrap, tracked by the barrier; J rows by bulk copies
      for (int c = 0; c < 3; ++c) {
        async_row(st + c * WE, is.e[c] + rofs, Es, WE, is.n1, lane);
        if (hasB) async_row(st + 3 * WE + c * WB, is.b[c] + rofs, Bs, WB, is.n1, lane);
      }
      cp_async_track(bar);
      if (lane == 0) slot_item[rc.islot] = ik;
      __syncwarp();
      if (lane == 0) mbar_expect_tx(bar, (uint32_t)((hasJ ? 3 * SWc : 0) * sizeof(T)));
      __syncwarp();
      if (lane >= 6 && lane < 9 && hasJ)
        bulk_g2s(st + 3 * WE + 3 * WB + c3 * SW, is.j[c3] + (int64_t)t * is.p1 + is.i0,
                 (uint32_t)(SWc * sizeof(T)), bar);
    }
    __syncwarp();
    ++rc.inflight;
    if (++rc.islot == NS) rc.islot = 0;
    if (++iq == is.Rr + 2) {
      iq = 0;
      ik = take_item<T>(A, ctr, step, lane);
      if (ik >= 0) strip_item<T, MT>(A, ik, step, is);
    }
  };
  auto ready = [&]() -> bool {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[rc.wslot], (rc.wpar >> rc.wslot) & 1u,
                                                      limit_ns));
    if (!ok) {
      if (lane == 0) atomicOr(A.err, ERRBIT_TIMEOUT);
      int sl = rc.wslot;
      unsigned par = rc.wpar;
      for (int m = 0; m < rc.inflight; ++m) {
        mbar_wait(&bars[sl], (par >> sl) & 1u, limit_ns);
        par ^= 1u << sl;
        if (++sl == NS) sl = 0;
      }
      return false;
    }
    rc.wpar ^= 1u << rc.wslot;
    if (++rc.wslot == NS) rc.wslot = 0;
    --rc.inflight;
    return true;
  };

  for (int k = 0; k < NS; ++k) issue();
  while (rc.inflight > 0) {
    StripItem<T> it;
    strip_item<T, MT>(A, slot_item[rc.wslot], step, it);
    int cslot = rc.wslot;
    if (!ready()) return false;
    for (int q = 0; q <= it.Rr; ++q) {
      const int nslot = rc.wslot;
      if (!ready()) return false;
      const T* sq = wbase + cslot * A.sh.stage_elems;
      const T* sq1 = wbase + nslot * A.sh.stage_elems;
      march_row<T, MT>(sq, sq1, bnew, q, it.r0 - 1 + q, it.i0, it.n1, it.p1, A.gh, WE, WB, SW, s,
                       dt, it.eo, it.bo, has_j, has_j ? it.j : nullptr, lane);
      fence_proxy_async();
      __syncwarp();
      issue();
      cslot = nslot;
    }
    issue();
  }
  return true;
}

template <typename T, int MT>
__global__ void __launch_bounds__(256, 1) batch_kernel(BatchArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ StencilArgs<T> s_sten;   // the particle path takes its address
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int NS = A.sh.NS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw) + wib * NS;
  int* slot_item = reinterpret_cast<int*>(smem_raw + (size_t)nw * NS * 8) + wib * NS;
  T* wbase = reinterpret_cast<T*>(smem_raw + A.sh.hdr_bytes) + (size_t)wib * A.sh.warp_elems;
  if (threadIdx.x == 0) s_sten = A.s;
  if (lane == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k]);
    mbar_init_fence();
  }
  __syncthreads();
  const int gw = blockIdx.x * nw + wib, tw = gridDim.x * nw;
  const int npitems = A.nitems - A.nfield - A.ncorr;
  RingCursor rc{0, 0, 0, 0u};
  bool ok = true;
  unsigned epoch = 0;
  // particles | x1 current correction | fields, a grid barrier after each
  const int nphase = A.has_current ? (A.ncorr ? 3 : 2) : 1;
  for (int64_t step = 0; step < A.max_steps; ++step) {
    // the counter of the next step was last used before the previous barrier
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(A.ctr + ((step + 1) & 1), 0u);
    for (int phase = 0; phase < nphase; ++phase) {
      if (phase == 0) {
        for (int k = gw; k < npitems; k += tw) {
          const int2 w = A.items[A.nfield + k];
          const RunInfo R = A.runs[w.x];
          if (step >= R.nsteps) continue;
          particle_chunk<T>(A, &s_sten, R, w.y, (R.cur + (int)step) & 1, lane);
        }
      }
      if (phase == 1 && nphase == 3) {
        for (int k = gw; k < A.ncorr; k += tw) {
          const int2 w = A.items[A.nitems - A.ncorr + k];
          const RunInfo R = A.runs[w.x];
          if (step >= R.nsteps) continue;
          correct_row<T>(A, R, w.y, wbase, lane);
        }
      }
      if (ok && phase == nphase - 1)
        ok = field_phase<T, MT>(A, A.s, step, bars, slot_item, wbase, rc, lane);
      // this step's stores are read by bulk copies after the barrier
      fence_proxy_async_global();
      if (!grid_wait(A, epoch)) return;
      if (*((volatile unsigned*)A.err) & ERRBIT_TIMEOUT) return;
    }
  }
}

// Laser fields of one run (E2 and B3 of the x1 eigenmode profile times the
// Gaussian transverse factor, as the single-run laser load), rows p1 apart;
// the other components are cleared.
template <typename T>
__global__ void run_laser_kernel(T* e1, T* e2, T* e3, T* b1, T* b2, T* b3, int n1, int n2, int p1,
                                 int gh, double dx2, const double* ep, const double* bp,
                                 double w0, double x2c) {
  // every column c in [-gh, n1 + gh) of each row, ghosts holding column c mod n1
  const int w = n1 + 2 * gh;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)w * n2;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % w) - gh, j = (int)(q / w);
    const int i = wrap_index(c, n1);
    double tr = 1.0;
    if (w0 > 0.0) {
      const double d2 = ((j + 0.5) * dx2 - x2c) / w0;  // E2 and B3 sit at x2 = (j+1/2) dx2
      tr = exp(-d2 * d2);
    }
    const int64_t k = (int64_t)j * p1 + c;
    e1[k] = (T)0;
    e3[k] = (T)0;
    b1[k] = (T)0;
    b2[k] = (T)0;
    e2[k] = (T)(ep[i] * tr);
    b3[k] = (T)(bp[i] * tr);
  }
}

template <typename T>
using BatchKernel = void (*)(BatchArgs<T>);

// the persistent kernel unrolled for the stencil reach of M taps
template <typename T>
BatchKernel<T> batch_kernel_for(int M) {
  switch (stencil_mt(M)) {
    case 8:
      return batch_kernel<T, 8>;
    case 16:
      return batch_kernel<T, 16>;
    default:
      return batch_kernel<T, 32>;
  }
}

template <typename T>
__global__ void commit_parity_kernel(RunInfo* runs, int nruns) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nruns; r += gridDim.x * blockDim.x)
    runs[r].cur = (runs[r].cur + (int)(runs[r].nsteps & 1)) & 1;
}

}  // namespace

struct pic_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nruns = 0;
  int64_t cells = 0;  // sum over runs of n1*n2 (pool arrays are padded per run)
  int precision = PIC_MIXED, pusher = PIC_ANALYTIC;
  size_t tsize = 4;
  double dt = 0, dx[2] = {0, 0};
  int M = 0;
  double cE[PIC_MAX_M] = {0}, cB[PIC_MAX_M] = {0};
  StencilArgs<double> sd{};
  StencilArgs<float> sf{};
  StencilArgs<dfl> sdf{};
  std::vector<RunInfo> runs;
  int64_t total = 0;
  void* pool = nullptr;
  RunInfo* d_runs = nullptr;
  int2* d_items = nullptr;
  int nitems = 0, items_cap = 0;
  PartPtrs parts{};
  int64_t np = 0;
  double qm = -1.0;
  int has_current = 0;
  int sw = 224, rows = 16, stages = 2, warps = 2;  // field strips (see StripShape)
  int gh = 0;  // ghost columns on each side of a pool row
  int nfield = 0;
  int corr = 0;              // C^B != e_1: the x1 current correction runs with the deposit
  void* taps = nullptr;      // correction taps of every row length, field precision
  int corr_elems = 0;        // shared-memory elements a warp needs for one corrected row
  int ncorr = 0;
  unsigned* bar = nullptr;
  unsigned* ctr = nullptr;
  unsigned* err = nullptr;
  double timeout_s = 5.0;
  int impossible = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_dirty = true;
  bool used_graph = false;
  int grid = 0, bps = 0;
  size_t smem = 0;
  int64_t max_steps = 0;
  float last_ms = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::string msg;
};

namespace {

pic_status bfail(pic_batch* b, pic_status s, const std::string& m) {
  if (b) b->msg = m;
  return s;
}

#define BCK(b, call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      (b)->msg = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA;        \
    }                                                                             \
  } while (0)

template <typename T>
void fill_stencil_b(pic_batch* b, StencilArgs<T>& s) {
  s.M = b->M;
  for (int j = 0; j < PIC_MAX_M; ++j) {
    s.kE[j] = (T)(j < b->M ? b->dt * b->cE[j] / b->dx[0] : 0.0);
    s.kB[j] = (T)(j < b->M ? b->dt * b->cB[j] / b->dx[0] : 0.0);
  }
  s.y2 = (T)(b->dt / b->dx[1]);
  s.y3 = (T)0;
}

StripShape strip_shape(const pic_batch* b) {
  const int V = 16 / (int)b->tsize;
  const Reach R(stencil_mt(b->M), V);
  StripShape sh;
  sh.SW = b->sw;
  sh.R = b->rows;
  sh.NS = b->stages;
  sh.NW = b->warps;
  sh.WE = R.WE(sh.SW, V);
  sh.WB = R.WB(sh.SW, V);
  sh.stage_elems = 3 * (sh.WE + sh.WB + sh.SW);
  sh.warp_elems = std::max(sh.NS * sh.stage_elems + 6 * sh.WB, b->corr_elems);
  sh.hdr_bytes = (sh.NW * sh.NS * 12 + 127) / 128 * 128;  // mbarriers + stage item ids
  return sh;
}

size_t strip_smem_bytes(const pic_batch* b) {
  const StripShape sh = strip_shape(b);
  return sh.hdr_bytes + (size_t)sh.NW * sh.warp_elems * b->tsize;
}

// work items for the current strip shape and particle set: field strips of all
// runs (x1 strip fastest), then 32-particle chunks
pic_status build_items(pic_batch* b) {
  std::vector<int2> items;
  for (int r = 0; r < b->nruns; ++r) {
    RunInfo& R = b->runs[r];
    R.nstrips = (R.n1 + b->sw - 1) / b->sw;
    const int nf = R.nstrips * ((R.n2 + b->rows - 1) / b->rows);
    for (int t = 0; t < nf; ++t) items.push_back(make_int2(r, t));
  }
  b->nfield = (int)items.size();
  for (int r = 0; r < b->nruns; ++r) {
    const RunInfo& R = b->runs[r];
    const int64_t n = R.p1 - R.p0;
    const int chunks = (int)((n + 31) / 32);
    for (int c = 0; c < chunks; ++c) items.push_back(make_int2(r, c));
  }
  b->ncorr = 0;
  if (b->corr && b->has_current) {
    for (int r = 0; r < b->nruns; ++r)
      for (int j = 0; j < b->runs[r].n2; ++j) items.push_back(make_int2(r, j));
    int64_t nc = 0;
    for (int r = 0; r < b->nruns; ++r) nc += b->runs[r].n2;
    b->ncorr = (int)nc;
  }
  if ((int)items.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    BCK(b, cudaMalloc(&b->d_items, sizeof(int2) * items.size()));
    b->items_cap = (int)items.size();
  }
  b->nitems = (int)items.size();
  BCK(b, cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  BCK(b, cudaMemcpy(b->d_runs, b->runs.data(), sizeof(RunInfo) * b->nruns, cudaMemcpyHostToDevice));
  b->graph_dirty = true;
  return PIC_OK;
}

template <typename T>
const StencilArgs<T>& stencil_of(const pic_batch* b);
template <>
const StencilArgs<double>& stencil_of<double>(const pic_batch* b) { return b->sd; }
template <>
const StencilArgs<float>& stencil_of<float>(const pic_batch* b) { return b->sf; }
template <>
const StencilArgs<dfl>& stencil_of<dfl>(const pic_batch* b) { return b->sdf; }

template <typename T>
pic_status launch_batch(pic_batch* b) {
  BatchArgs<T> A;
  A.runs = b->d_runs;
  A.items = b->d_items;
  A.nitems = b->nitems;
  A.pool = (T*)b->pool;
  A.total = b->total;
  A.parts = b->parts;
  A.s = stencil_of<T>(b);
  memset(&A.gbase, 0, sizeof A.gbase);
  A.gbase.ndim = 2;
  for (int d = 0; d < 2; ++d) {
    A.gbase.dx[d] = b->dx[d];
    A.gbase.inv_dx[d] = 1.0 / b->dx[d];
    A.gbase.dx_dt[d] = b->dx[d] / b->dt;
  }
  A.gbase.dx[2] = 1.0;
  A.gbase.inv_dx[2] = 1.0;
  A.gbase.n[2] = 1;
  A.gbase.dt = b->dt;
  A.a = PartArgs{b->qm, b->pusher, b->np};
  A.sh = strip_shape(b);
  A.gh = b->gh;
  A.nfield = b->nfield;
  A.ncorr = b->ncorr;
  A.taps = (const T*)b->taps;
  A.ctr = b->ctr;
  A.max_steps = b->max_steps;
  A.has_current = b->has_current;
  A.bar = b->bar;
  A.err = b->err;
  A.timeout_ns = (long long)(b->timeout_s * 1e9);
  b->smem = A.sh.hdr_bytes + (size_t)A.sh.NW * A.sh.warp_elems * sizeof(T);
  const BatchKernel<T> kern = batch_kernel_for<T>(b->M);
  BCK(b, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int nsm = 0, bps = 0;
  BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
  BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 32 * A.sh.NW, b->smem));
  if (bps < 1) return bfail(b, PIC_ERR_CUDA, "persistent kernel does not fit on an SM");
  b->bps = bps;
  b->grid = std::max(1, bps * nsm);
  A.expected = (unsigned)b->grid + (b->impossible ? 1u : 0u);

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(32 * A.sh.NW);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;

  auto enqueue = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->ctr, 0, 2 * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return e;
    e = cudaLaunchKernelEx(&cfg, kern, A);
    if (e != cudaSuccess) return e;
    commit_parity_kernel<T><<<(b->nruns + 255) / 256, 256, 0, b->stream>>>(b->d_runs, b->nruns);
    return cudaGetLastError();
  };
  if (b->graph_dirty) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = enqueue();
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
          cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess) {
        b->graph_dirty = false;
      } else {
        b->graph = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // a failed capture leaves no sticky error
  }
  BCK(b, cudaEventRecord(b->ev[0], b->stream));
  if (b->graph) {
    b->used_graph = true;
    BCK(b, cudaGraphLaunch(b->graph, b->stream));
  } else {
    b->used_graph = false;
    BCK(b, enqueue());
  }
  BCK(b, cudaEventRecord(b->ev[1], b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, cudaEventElapsedTime(&b->last_ms, b->ev[0], b->ev[1]));
  unsigned h = 0;
  BCK(b, cudaMemcpy(&h, b->err, sizeof h, cudaMemcpyDeviceToHost));
  BCK(b, cudaMemcpy(b->runs.data(), b->d_runs, sizeof(RunInfo) * b->nruns, cudaMemcpyDeviceToHost));
  if (h) {
    BCK(b, cudaMemset(b->err, 0, sizeof(unsigned)));
    if (h & ERRBIT_TIMEOUT) return bfail(b, PIC_ERR_TIMEOUT, "grid barrier wait timed out");
    return bfail(b, PIC_ERR_DEVICE_CHECK, "device check failed in the ensemble kernel");
  }
  return PIC_OK;
}

pic_status run_now(pic_batch* b) {
  int64_t mx = 0;
  for (const RunInfo& R : b->runs) mx = std::max(mx, R.nsteps);
  if (mx != b->max_steps) b->graph_dirty = true;
  b->max_steps = mx;
  if (b->precision == PIC_FP64) return launch_batch<double>(b);
  if (b->precision == PIC_COMPENSATED) return launch_batch<dfl>(b);
  return launch_batch<float>(b);
}

}  // namespace

extern "C" {

pic_status pic_batch_init(const pic_batch_desc* d, double dt, const pic_coeffs* co, void* stream,
                          pic_batch** out) {
  if (!out) return PIC_ERR_ARG;
  *out = nullptr;
  if (!d || !co || d->nruns < 1 || !d->n1 || !d->n2 || !(dt > 0)) return PIC_ERR_ARG;
  if (d->precision != PIC_FP64 && d->precision != PIC_MIXED && d->precision != PIC_COMPENSATED)
    return PIC_ERR_ARG;
  if (d->pusher != PIC_BORIS && d->pusher != PIC_ANALYTIC && d->pusher != PIC_HC)
    return PIC_ERR_ARG;
  if (co->M < 1 || co->M > PIC_MAX_M || !co->cE || !co->cB) return PIC_ERR_ARG;
  if (!(d->dx[0] > 0) || !(d->dx[1] > 0)) return PIC_ERR_ARG;
  for (int r = 0; r < d->nruns; ++r)
    if (d->n1[r] < 1 || d->n2[r] < 1) return PIC_ERR_ARG;
  pic_batch* b = new pic_batch();
  b->nruns = d->nruns;
  b->precision = d->precision;
  b->pusher = d->pusher;
  b->tsize = d->precision == PIC_MIXED ? 4 : 8;  // FP32, or FP64 / an FP32 pair
  b->dt = dt;
  b->dx[0] = d->dx[0];
  b->dx[1] = d->dx[1];
  b->M = co->M;
  for (int j = 0; j < co->M; ++j) {
    b->cE[j] = co->cE[j];
    b->cB[j] = co->cB[j];
  }
  // exact CFL condition, Eq. (21): the x1 product is grid independent, the x2
  // Yee term is at most (2/dx2)^2 for every run
  {
    double pmax = 0, pmin = 0;
    for (int q = 0; q < 20001; ++q) {
      const double k = M_PI / b->dx[0] * q / 20000.0;
      const double p = host_kspace(b->M, b->cB, k, b->dx[0]) * host_kspace(b->M, b->cE, k, b->dx[0]);
      pmax = std::max(pmax, p);
      pmin = std::min(pmin, p);
    }
    const double lhs = (dt / 2) * (dt / 2) * (pmax + (2.0 / b->dx[1]) * (2.0 / b->dx[1]));
    if (lhs > 1.0 + 1e-12 || pmin < -1e-12 * std::max(pmax, 1e-300)) {
      delete b;
      return PIC_ERR_CFL;
    }
  }
  b->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return PIC_ERR_CUDA;
  }
  b->runs.resize(b->nruns);
  {
    // ghost width: the reach of the unrolled x1 stencils on both sides
    const int V = 16 / (int)b->tsize;
    const Reach R(stencil_mt(b->M), V);
    b->gh = R.DB + R.DE;
  }
  int64_t off = 0;
  for (int r = 0; r < b->nruns; ++r) {
    if (d->n1[r] < 1 || d->n2[r] < 1) {
      delete b;
      return PIC_ERR_ARG;
    }
    RunInfo& R = b->runs[r];
    // rows carry gh ghost columns on each side and are padded to 16 bytes; runs
    // start on 256-byte boundaries in every pool array (vector and bulk accesses)
    const int V = 16 / (int)b->tsize;
    const int ld = (d->n1[r] + 2 * b->gh + V - 1) / V * V;
    R = RunInfo{d->n1[r], d->n2[r], ld, off, 0, 0, 0, 0, 0};
    off += ((int64_t)ld * d->n2[r] + 63) / 64 * 64;
    b->cells += (int64_t)d->n1[r] * d->n2[r];
  }
  b->total = off;
  fill_stencil_b<double>(b, b->sd);
  fill_stencil_b<float>(b, b->sf);
  fill_stencil_b<dfl>(b, b->sdf);
  b->sw = b->tsize == 4 ? 224 : 160;
  b->rows = b->tsize == 4 ? 16 : 32;
  b->stages = 2;
  b->warps = 2;
  auto init_fail = [&](pic_status s) {
    pic_batch_destroy(b);
    return s;
  };
  if (cudaMalloc(&b->pool, b->tsize * b->total * 15) != cudaSuccess) return init_fail(PIC_ERR_OOM);
  if (cudaMemsetAsync(b->pool, 0, b->tsize * b->total * 15, b->stream) != cudaSuccess ||
      cudaMalloc(&b->d_runs, sizeof(RunInfo) * b->nruns) != cudaSuccess ||
      cudaMalloc(&b->bar, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->ctr, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->err, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(b->err, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess)
    return init_fail(PIC_ERR_CUDA);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return init_fail(PIC_ERR_CUDA);
  // x1 current correction (Sec. 3.3): one tap set per distinct row length
  for (int j = 0; j < b->M; ++j)
    if (b->cB[j] != (j == 0 ? 1.0 : 0.0)) b->corr = 1;
  if (b->corr) {
    std::vector<double> all;
    std::vector<int> seen_n1, seen_off, seen_cnt, seen_lo;
    const int V = 16 / (int)b->tsize;
    for (int r = 0; r < b->nruns; ++r) {
      RunInfo& R = b->runs[r];
      size_t k = 0;
      while (k < seen_n1.size() && seen_n1[k] != R.n1) ++k;
      if (k == seen_n1.size()) {
        std::vector<double> taps;
        int lo = 0;
        if (!inv_circulant_taps(R.n1, b->dx[0], b->M, b->cB, taps, lo)) {
          b->msg = "C^B gives [k]_B1 = 0 at a grid mode";
          return init_fail(PIC_ERR_ARG);
        }
        seen_n1.push_back(R.n1);
        seen_off.push_back((int)all.size());
        seen_cnt.push_back((int)taps.size());
        seen_lo.push_back(lo);
        all.insert(all.end(), taps.begin(), taps.end());
        all.resize(ceil_to((int)all.size(), V), 0.0);  // every tap set 16-byte aligned
      }
      R.toff = seen_off[k];
      R.tcount = seen_cnt[k];
      R.tlo = seen_lo[k];
      b->corr_elems = std::max(b->corr_elems, ceil_to(R.n1, V) + 2 * ceil_to(R.tcount, V));
    }
    bool ok;
    if (b->precision == PIC_FP64) {
      ok = cudaMalloc(&b->taps, sizeof(double) * all.size()) == cudaSuccess &&
           cudaMemcpy(b->taps, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice) ==
               cudaSuccess;
    } else if (b->precision == PIC_COMPENSATED) {
      std::vector<dfl> td;
      for (double v : all) td.push_back(dfl(v));
      ok = cudaMalloc(&b->taps, sizeof(dfl) * td.size()) == cudaSuccess &&
           cudaMemcpy(b->taps, td.data(), sizeof(dfl) * td.size(), cudaMemcpyHostToDevice) ==
               cudaSuccess;
    } else {
      std::vector<float> tf(all.begin(), all.end());
      ok = cudaMalloc(&b->taps, sizeof(float) * tf.size()) == cudaSuccess &&
           cudaMemcpy(b->taps, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice) ==
               cudaSuccess;
    }
    if (!ok) return init_fail(PIC_ERR_CUDA);
    if (strip_smem_bytes(b) > 200 * 1024) {
      b->msg = "an x1 row and its correction taps do not fit in a warp's shared memory";
      return init_fail(PIC_ERR_ARG);
    }
  }
  if (build_items(b) != PIC_OK) return init_fail(PIC_ERR_CUDA);
  *out = b;
  return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch* b) {
  if (!b) return PIC_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->pool);
  cudaFree(b->taps);
  cudaFree(b->d_runs);
  cudaFree(b->d_items);
  cudaFree(b->bar);
  cudaFree(b->ctr);
  cudaFree(b->err);
  for (int d = 0; d < 3; ++d) {
    cudaFree(b->parts.x[d]);
    cudaFree(b->parts.u[d]);
  }
  cudaFree(b->parts.w);
  if (b->ev[0]) cudaEventDestroy(b->ev[0]);
  if (b->ev[1]) cudaEventDestroy(b->ev[1]);
  delete b;
  return PIC_OK;
}

const char* pic_batch_last_error(const pic_batch* b) { return b ? b->msg.c_str() : ""; }

pic_status pic_batch_load_laser(pic_batch* b, const pic_laser* L) {
  if (!b || !L) return bfail(b, PIC_ERR_ARG, "null argument");
  BCK(b, cudaSetDevice(b->device));
  int nmax = 0;
  for (const RunInfo& R : b->runs) nmax = std::max(nmax, R.n1);
  double* dev = nullptr;
  BCK(b, cudaMalloc(&dev, sizeof(double) * 2 * nmax));
  std::vector<double> ep(nmax), bp(nmax);
  pic_status st = PIC_OK;
  for (int r = 0; r < b->nruns && st == PIC_OK; ++r) {
    RunInfo& R = b->runs[r];
    const pic_laser& l = L[r];
    if (!(l.L_env > 0) || l.L_env > R.n1 * b->dx[0] || !(l.k0 > 0) || !isfinite(l.a0)) {
      st = bfail(b, PIC_ERR_ARG, "laser envelope must fit the run's box");
      break;
    }
    laser_profiles(R.n1, b->dx[0], b->dt, b->M, b->cE, b->cB, l, ep.data(), bp.data());
    cudaError_t e = cudaMemcpy(dev, ep.data(), sizeof(double) * R.n1, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dev + R.n1, bp.data(), sizeof(double) * R.n1, cudaMemcpyHostToDevice);
    const int par = R.cur;
    if (e == cudaSuccess) {
      const unsigned nb =
          (unsigned)std::min<int64_t>(((int64_t)(R.n1 + 2 * b->gh) * R.n2 + 255) / 256, 4096);
      if (b->precision == PIC_FP64) {
        double* f[6];
        for (int c = 0; c < 6; ++c)
          f[c] = (double*)b->pool + (int64_t)(par * 6 + c) * b->total + R.off + b->gh;
        run_laser_kernel<double><<<nb, 256, 0, b->stream>>>(f[0], f[1], f[2], f[3], f[4], f[5], R.n1,
                                                            R.n2, R.ld, b->gh, b->dx[1], dev, dev + R.n1,
                                                            l.w0, l.x2c);
      } else if (b->precision == PIC_COMPENSATED) {
        dfl* f[6];
        for (int c = 0; c < 6; ++c)
          f[c] = (dfl*)b->pool + (int64_t)(par * 6 + c) * b->total + R.off + b->gh;
        run_laser_kernel<dfl><<<nb, 256, 0, b->stream>>>(f[0], f[1], f[2], f[3], f[4], f[5], R.n1,
                                                         R.n2, R.ld, b->gh, b->dx[1], dev, dev + R.n1,
                                                         l.w0, l.x2c);
      } else {
        float* f[6];
        for (int c = 0; c < 6; ++c)
          f[c] = (float*)b->pool + (int64_t)(par * 6 + c) * b->total + R.off + b->gh;
        run_laser_kernel<float><<<nb, 256, 0, b->stream>>>(f[0], f[1], f[2], f[3], f[4], f[5], R.n1,
                                                           R.n2, R.ld, b->gh, b->dx[1], dev, dev + R.n1,
                                                           l.w0, l.x2c);
      }
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaFree(dev);
  return st;
}

pic_status pic_batch_load_particles(pic_batch* b, const int64_t* counts, const double* x,
                                    const double* u, const double* w, double qm) {
  if (!b || !counts) return bfail(b, PIC_ERR_ARG, "null argument");
  BCK(b, cudaSetDevice(b->device));
  int64_t n = 0;
  for (int r = 0; r < b->nruns; ++r) {
    if (counts[r] < 0) return bfail(b, PIC_ERR_ARG, "negative count");
    n += counts[r];
  }
  if (n > 0 && (!x || !u || !w)) return bfail(b, PIC_ERR_ARG, "null particle arrays");
  int64_t p = 0;
  int hc = 0;
  for (int r = 0; r < b->nruns; ++r) {
    RunInfo& R = b->runs[r];
    R.p0 = p;
    R.p1 = p + counts[r];
    for (int64_t q = R.p0; q < R.p1; ++q) {
      if (!(x[q] >= 0 && x[q] < R.n1 * b->dx[0]) || !(x[n + q] >= 0 && x[n + q] < R.n2 * b->dx[1]))
        return bfail(b, PIC_ERR_ARG, "particle outside its run's box");
      if (w[q] != 0.0) hc = 1;
    }
    p = R.p1;
  }
  for (int d = 0; d < 3; ++d) {
    cudaFree(b->parts.x[d]);
    cudaFree(b->parts.u[d]);
    b->parts.x[d] = b->parts.u[d] = nullptr;
  }
  cudaFree(b->parts.w);
  b->parts.w = nullptr;
  b->np = n;
  b->qm = qm;
  b->has_current = hc;
  if (n > 0) {
    for (int d = 0; d < 2; ++d) {
      BCK(b, cudaMalloc(&b->parts.x[d], sizeof(double) * n));
      BCK(b, cudaMemcpy(b->parts.x[d], x + d * n, sizeof(double) * n, cudaMemcpyHostToDevice));
    }
    for (int d = 0; d < 3; ++d) {
      BCK(b, cudaMalloc(&b->parts.u[d], sizeof(double) * n));
      BCK(b, cudaMemcpy(b->parts.u[d], u + d * n, sizeof(double) * n, cudaMemcpyHostToDevice));
    }
    BCK(b, cudaMalloc(&b->parts.w, sizeof(double) * n));
    BCK(b, cudaMemcpy(b->parts.w, w, sizeof(double) * n, cudaMemcpyHostToDevice));
  }
  return build_items(b);
}

pic_status pic_batch_set_steps(pic_batch* b, const int64_t* nsteps) {
  if (!b || !nsteps) return bfail(b, PIC_ERR_ARG, "null argument");
  for (int r = 0; r < b->nruns; ++r) {
    if (nsteps[r] < 0) return bfail(b, PIC_ERR_ARG, "negative step count");
    b->runs[r].nsteps = nsteps[r];
  }
  BCK(b, cudaSetDevice(b->device));
  BCK(b, cudaMemcpy(b->d_runs, b->runs.data(), sizeof(RunInfo) * b->nruns, cudaMemcpyHostToDevice));
  b->graph_dirty = true;
  return PIC_OK;
}

pic_status pic_batch_run(pic_batch* b) {
  if (!b) return PIC_ERR_ARG;
  BCK(b, cudaSetDevice(b->device));
  return run_now(b);
}

pic_status pic_batch_autotune(pic_batch* b, int trial_steps) {
  if (!b || trial_steps < 1) return bfail(b, PIC_ERR_ARG, "trial_steps must be >= 1");
  BCK(b, cudaSetDevice(b->device));
  // field strips: (x1 columns, rows per item, ring stages, warps per CTA)
  static const int cand32[][4] = {{224, 16, 2, 2}, {224, 32, 2, 2}, {288, 16, 2, 2},
                                  {352, 16, 3, 2}, {160, 32, 2, 2}, {128, 32, 2, 2}};
  static const int cand64[][4] = {{96, 32, 2, 2}, {160, 32, 2, 2}, {224, 32, 2, 2},
                                  {160, 16, 3, 2}};
  const int (*cand)[4] = b->tsize == 4 ? cand32 : cand64;
  const int ncand = b->tsize == 4 ? 6 : 4;
  std::vector<int64_t> saved(b->nruns);
  for (int r = 0; r < b->nruns; ++r) {
    saved[r] = b->runs[r].nsteps;
    b->runs[r].nsteps = trial_steps;
  }
  float best = 1e30f;
  int bc[4] = {b->sw, b->rows, b->stages, b->warps};
  pic_status st = PIC_OK;
  for (int c = 0; c < ncand && st == PIC_OK; ++c) {
    b->sw = cand[c][0];
    b->rows = cand[c][1];
    b->stages = cand[c][2];
    b->warps = cand[c][3];
    if (strip_smem_bytes(b) > 200 * 1024) continue;
    st = build_items(b);
    if (st == PIC_OK) st = run_now(b);
    if (st == PIC_OK && b->last_ms < best) {
      best = b->last_ms;
      for (int k = 0; k < 4; ++k) bc[k] = cand[c][k];
    }
  }
  b->sw = bc[0];
  b->rows = bc[1];
  b->stages = bc[2];
  b->warps = bc[3];
  for (int r = 0; r < b->nruns; ++r) {
    b->runs[r].nsteps = saved[r];
    b->runs[r].cur = 0;
  }
  BCK(b, cudaMemset(b->pool, 0, b->tsize * b->total * 15));
  pic_status st2 = build_items(b);
  return st != PIC_OK ? st : st2;
}

pic_status pic_batch_read_particles(pic_batch* b, double* x, double* u, double* w) {
  if (!b) return PIC_ERR_ARG;
  BCK(b, cudaSetDevice(b->device));
  const int64_t n = b->np;
  if (n == 0) return PIC_OK;
  for (int d = 0; d < 2 && x; ++d)
    BCK(b, cudaMemcpy(x + d * n, b->parts.x[d], sizeof(double) * n, cudaMemcpyDeviceToHost));
  for (int d = 0; d < 3 && u; ++d)
    BCK(b, cudaMemcpy(u + d * n, b->parts.u[d], sizeof(double) * n, cudaMemcpyDeviceToHost));
  if (w) BCK(b, cudaMemcpy(w, b->parts.w, sizeof(double) * n, cudaMemcpyDeviceToHost));
  return PIC_OK;
}

pic_status pic_batch_read_field(pic_batch* b, int run, int comp, double* buf) {
  if (!b || !buf || run < 0 || run >= b->nruns || comp < 0 || comp > PIC_J3)
    return bfail(b, PIC_ERR_ARG, "bad run, component or buffer");
  BCK(b, cudaSetDevice(b->device));
  const RunInfo& R = b->runs[run];
  const int slot = comp < 6 ? R.cur * 6 + comp : 12 + (comp - 6);
  const int64_t n = (int64_t)R.n1 * R.n2;
  const char* src =
      (const char*)b->pool + ((int64_t)slot * b->total + R.off + b->gh) * b->tsize;
  // rows lie R.ld values apart in the pool, after gh ghost columns
  if (b->precision == PIC_FP64) {
    BCK(b, cudaMemcpy2D(buf, sizeof(double) * R.n1, src, sizeof(double) * R.ld,
                        sizeof(double) * R.n1, R.n2, cudaMemcpyDeviceToHost));
  } else if (b->precision == PIC_COMPENSATED) {
    std::vector<dfl> tmp(n);
    BCK(b, cudaMemcpy2D(tmp.data(), sizeof(dfl) * R.n1, src, sizeof(dfl) * R.ld,
                        sizeof(dfl) * R.n1, R.n2, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) buf[i] = (double)tmp[i];
  } else {
    std::vector<float> tmp(n);
    BCK(b, cudaMemcpy2D(tmp.data(), sizeof(float) * R.n1, src, sizeof(float) * R.ld,
                        sizeof(float) * R.n1, R.n2, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) buf[i] = tmp[i];
  }
  return PIC_OK;
}

pic_status pic_batch_get_info(pic_batch* b, pic_batch_info* info) {
  if (!b || !info) return bfail(b, PIC_ERR_ARG, "null argument");
  memset(info, 0, sizeof *info);
  info->tile[0] = b->sw;
  info->tile[1] = b->rows;
  info->grid_blocks = b->grid;
  info->blocks_per_sm = b->bps;
  info->work_items = b->nitems;
  info->graph = b->used_graph ? 1 : 0;
  info->total_cells = b->cells;
  info->max_steps = b->max_steps;
  for (const RunInfo& R : b->runs) {
    info->cell_steps += (int64_t)R.n1 * R.n2 * R.nsteps;
    info->particle_steps += (R.p1 - R.p0) * R.nsteps;
  }
  info->last_run_ms = b->last_ms;
  info->has_current = b->has_current;
  info->correction_active = b->ncorr > 0 ? 1 : 0;
  return PIC_OK;
}

pic_status pic_batch_set_strip(pic_batch* b, int width, int rows, int stages, int warps) {
  if (!b) return PIC_ERR_ARG;
  const int V = 16 / (int)b->tsize;
  if (width < V || width % V != 0 || width > 4096 || rows < 1 || stages < 2 || stages > 8 ||
      warps < 1 || warps > 8)
    return bfail(b, PIC_ERR_ARG,
                 "strip width a positive multiple of 16 bytes, rows >= 1, 2 <= stages <= 8, "
                 "1 <= warps <= 8");
  const int keep[4] = {b->sw, b->rows, b->stages, b->warps};
  b->sw = width;
  b->rows = rows;
  b->stages = stages;
  b->warps = warps;
  if (strip_smem_bytes(b) > 200 * 1024) {
    b->sw = keep[0];
    b->rows = keep[1];
    b->stages = keep[2];
    b->warps = keep[3];
    return bfail(b, PIC_ERR_ARG, "strip rows do not fit in shared memory");
  }
  BCK(b, cudaSetDevice(b->device));
  return build_items(b);
}

pic_status pic_batch_set_barrier(pic_batch* b, double timeout_s, int impossible) {
  if (!b || !(timeout_s > 0)) return bfail(b, PIC_ERR_ARG, "timeout must be positive");
  b->timeout_s = timeout_s;
  b->impossible = impossible ? 1 : 0;
  b->graph_dirty = true;
  return PIC_OK;
}

}  // extern "C"
