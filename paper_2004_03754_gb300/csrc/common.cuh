// common.cuh -- shared device/host definitions of libpic (GB300, sm_103a).
//
// Layout of a context in HBM (all arrays separate allocations, 256-byte aligned):
//   fields   E1 E2 E3 B1 B2 B3 J1 J2 J3   n1*n2*n3 values of T (double or float), x1 fastest
//   particles x1 x2 [x3] u1 u2 u3 w (double) + id (int64), two copies (ping-pong for re-binning)
//   bins     per-tile counts and starts (int64), per-particle tile key and slot (int32)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "march_layout.cuh"
#include "pic.h"

namespace pic {

template <typename T>
struct FieldPtrs {
  T* e[3];
  T* b[3];  // B^{n-1/2}
  T* j[3];
};

// time-centred B^n arrays (3D: formed once per step before the particle tiles)
template <typename T>
struct BbarPtrs {
  T* b[3];
};

struct PartPtrs {
  double* x[3];
  double* u[3];
  double* w;
  int64_t* id;
  // energy-gain integrals of Sec. 4.2 per particle (W_LWFA, W_DLA); null when
  // the diagnostic is off
  double* wl;
  double* wd;
};

struct GridArgs {
  int ndim;
  int n[3];
  double dx[3];
  double inv_dx[3];
  double len[3];
  double dx_dt[3];   // dx_d / dt (Esirkepov running-sum factor)
  double dt;
  int64_t ncell;
};

// Stencil coefficients pre-multiplied by dt/dx1 (full step) in the field's type.
template <typename T>
struct StencilArgs {
  int M;
  T kE[PIC_MAX_M];   // dt * C^E_j / dx1
  T kB[PIC_MAX_M];   // dt * C^B_j / dx1
  T y2, y3;          // dt/dx2, dt/dx3 (Yee)
};

// Device error word bits (latched, read back by pic_sync / pic_read_*).
enum : unsigned {
  ERRBIT_MOVE = 1u,          // a particle moved a full cell or more in one step
  ERRBIT_ANALYTIC = 2u,      // the analytic pusher's proper-time iteration did not converge
  ERRBIT_NONFINITE = 4u,     // a non-finite momentum or position was produced
  ERRBIT_POSITION = 8u,      // a loaded particle position lies outside the box
  ERRBIT_TIMEOUT = 16u,      // a bounded wait (grid barrier, staging copy) ran out
};

__host__ __device__ inline int wrap_index(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// Launch helpers implemented in fields.cu / particles.cu (host side).
// ---------------------------------------------------------------------------
// Field tile shape and CTA size (threads 0 = 256); staging 0 = asynchronous bulk
// copies where the grid allows them (persistent kernels), 1 = synchronous loads
// only.  2D grids with bulk copies stream rows per warp instead: strips of sw x1
// columns and `rows` rows per work item, `warps` per CTA, a ring of `stages` rows.
struct FieldTile {
  int t[3];
  int threads;
  int staging;
  int sw, rows, warps, stages;
};

// Reads E^n, B^{n-1/2}, J from f; writes E^{n+1}, B^{n+1/2} into out.e / out.b.
// A staging wait that runs out latches ERRBIT_TIMEOUT in *err.
template <typename T>
cudaError_t launch_field_step(const FieldPtrs<T>& f, const FieldPtrs<T>& out, const GridArgs& g,
                              const StencilArgs<T>& s, const FieldTile& tile, unsigned* err,
                              cudaStream_t st);

template <typename T>
cudaError_t launch_bbar(const FieldPtrs<T>& f, const GridArgs& g, const StencilArgs<T>& s,
                        double* out, int comp, cudaStream_t st);

// path: 0 automatic, 1 whole rows in place, 2 row segments, 3 global memory
template <typename T>
cudaError_t launch_correct_j1(T* j1, T* tmp, const GridArgs& g, const T* taps, int lo, int count,
                              int path, cudaStream_t st);

template <typename T>
cudaError_t launch_convert_in(T* dst, const double* src, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_convert_out(double* dst, const T* src, int64_t n, cudaStream_t st);

template <typename T>
cudaError_t launch_laser_expand(const FieldPtrs<T>& f, const GridArgs& g, const double* eprof,
                                const double* bprof, double w0, double x2c, double x3c,
                                cudaStream_t st);

struct PartTile {
  int t[3];      // tile size in cells
  int g[3];      // guard cells of the staged window
  int nt[3];     // tiles per axis
  int64_t ntiles;
};

struct PartArgs {
  double qm;
  int pusher;
  int64_t np;
  // 1: the caller has formed the time-centred B in the BbarPtrs arrays (the
  // spectral field path); the particle kernels read it there in 2D and 3D
  int bbar_ready = 0;
};

struct BinBufs {
  int64_t* count;     // ntiles + 1 (the last bin holds particles being dropped)
  int64_t* start;     // ntiles + 2
  int* key;           // np
  int* slot;          // np
  int64_t* strag;     // np (indices of particles that take the global path)
  unsigned long long* strag_count;
  unsigned* err;
  int64_t* part;      // bin_scan_chunks(ntiles + 1): chunk sums of the scan
};

// chunks of the tile-count scan for n counts (the size of BinBufs::part)
int64_t bin_scan_chunks(int64_t n);


// kill_col >= 0: particles in x1 column kill_col are binned past the last tile
// (dropped by the caller); the count array holds ntiles + 1 bins
cudaError_t launch_bin_count(const PartPtrs& p, const GridArgs& g, const PartTile& t,
                             const BinBufs& b, int64_t np, cudaStream_t st, int kill_col = -1);
cudaError_t launch_bin_scan(const BinBufs& b, int64_t ntiles, cudaStream_t st);
cudaError_t launch_bin_scatter(const PartPtrs& src, const PartPtrs& dst, const GridArgs& g,
                               const BinBufs& b, int64_t np, cudaStream_t st);

template <typename T>
cudaError_t launch_particle_step(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                                 const GridArgs& g, const StencilArgs<T>& s, const PartTile& t,
                                 const PartArgs& a, const BinBufs& b, cudaStream_t st);

template <typename T>
cudaError_t launch_straggler_step(const FieldPtrs<T>& f, const BbarPtrs<T>& bg, const PartPtrs& p,
                                  const GridArgs& g, const StencilArgs<T>& s, const PartArgs& a,
                                  const BinBufs& b, int64_t max_count, cudaStream_t st);

// copy particles back in their original order; positions on the box edge are
// mapped into [0, len)
cudaError_t launch_unpermute(const PartPtrs& p, int ndim, int64_t np, double* x, double* u,
                             double* w, const double* len, cudaStream_t st);

// After particles were dropped: the kept ones (positions 0..kept-1, ids among
// 0..np_old-1) get ids 0..kept-1 in their old id order.  tmp: 2 np_old + 1 +
// bin_scan_chunks(np_old) values.
cudaError_t launch_renumber(int64_t* id, int64_t np_old, int64_t kept, int64_t* tmp,
                            cudaStream_t st);

// W_LWFA then W_DLA of every particle, in load order, into out (2 np values)
cudaError_t launch_unpermute_gain(const PartPtrs& p, int64_t np, double* out, cudaStream_t st);

size_t particle_smem_bytes(int ndim, size_t tsize, const PartTile& t, int M);

}  // namespace pic
