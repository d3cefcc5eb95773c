// particles.cu -- particle bookkeeping of libpic: binning by tile (counting
// sort), the read-back in load order and the shared-memory size of a tile.  The
// particle kernels themselves are in particle_kernels.cuh, compiled once per
// field type (particles_f32.cu, particles_f64.cu, particles_dfl.cu).
#include <math.h>

#include "common.cuh"
#include "fpbits.cuh"

namespace pic {

namespace {

// ---------------------------------------------------------------------------
// Binning (counting sort by tile)
// ---------------------------------------------------------------------------
// Particles of a warp are mostly in one tile (they were sorted by tile), so the
// lanes with equal keys take their slots from one counter update (a match over
// the warp, one atomic add of the group size by its first lane).  The cell floor
// is taken on the integer pipe (positions are in [0, L)).
__global__ void bin_count_kernel(PartPtrs p, GridArgs g, PartTile t, BinBufs b, int64_t np,
                                 int kill_col) {
  const unsigned lane = threadIdx.x & 31u;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
       q += (int64_t)gridDim.x * blockDim.x) {
    int tc[3] = {0, 0, 0}, c0 = 0;
    for (int d = 0; d < g.ndim; ++d) {
      int c = floor_pos(p.x[d][q] * g.inv_dx[d]);
      if (d == 0) c0 = c;
      c = c >= g.n[d] ? g.n[d] - 1 : c;
      tc[d] = c / t.t[d];
    }
    int key = (tc[2] * t.nt[1] + tc[1]) * t.nt[0] + tc[0];
    // the moving window's cleared column: its particles go to the bin after the
    // last tile, which the scatter places past the kept ones
    if (kill_col >= 0 && c0 == kill_col) key = (int)t.ntiles;
    b.key[q] = key;
    const unsigned peers = __match_any_sync(__activemask(), key);
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0ull;
    if ((int)lane == leader)
      base = atomicAdd((unsigned long long*)&b.count[key], (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    b.slot[q] = (int)(base + __popc(peers & ((1u << lane) - 1u)));
  }
}

// Exclusive scan of the n tile counts into start[0..n] (start[n] = total), in
// three passes over chunks of kScanChunk counts: chunk sums, a scan of the chunk
// sums by one CTA, then each chunk scanned from its offset.
constexpr int kScanT = 256, kScanPer = 8, kScanChunk = kScanT * kScanPer;

__global__ void __launch_bounds__(kScanT) bin_chunk_sum_kernel(BinBufs b, int64_t n) {
  __shared__ int64_t ws[kScanT / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < n) s += b.count[base + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kScanT / 32; ++w) t += ws[w];
    b.part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kScanT) bin_chunk_out_kernel(BinBufs b, int64_t n) {
  __shared__ int64_t ws[kScanT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  int64_t v[kScanPer], s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = base + k < n ? b.count[base + k] : 0;
    s += v[k];
  }
  // exclusive scan of the thread sums over the CTA
  int64_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  int64_t off = b.part[blockIdx.x];   // exclusive offset of the chunk
  for (int k = 0; k < w; ++k) off += ws[k];
  int64_t run = off + inc - s;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) b.start[base + k] = run;
    run += v[k];
  }
  if (base <= n - 1 && n - 1 < base + kScanPer) b.start[n] = run;   // the total
}

// exclusive scan of the m chunk sums in place (one CTA)
__global__ void __launch_bounds__(1024) bin_part_scan_kernel(BinBufs b, int64_t m) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  const int64_t per = (m + 1023) / 1024;
  const int64_t lo = tid * per, hi = (lo + per < m) ? lo + per : m;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += b.part[i];
  part[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t v = (tid >= off) ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int64_t run = part[tid] - s;  // exclusive prefix of this thread's chunk
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t c = b.part[i];
    b.part[i] = run;
    run += c;
  }
}

__global__ void bin_scatter_kernel(PartPtrs src, PartPtrs dst, int ndim, BinBufs b, int64_t np) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = b.start[b.key[q]] + b.slot[q];
    for (int d = 0; d < ndim; ++d) dst.x[d][o] = src.x[d][q];
    for (int c = 0; c < 3; ++c) dst.u[c][o] = src.u[c][q];
    dst.w[o] = src.w[q];
    dst.id[o] = src.id[q];
    if (src.wl) {
      dst.wl[o] = src.wl[q];
      dst.wd[o] = src.wd[q];
    }
  }
}

__global__ void unpermute_kernel(PartPtrs p, int ndim, int64_t np, double* x, double* u,
                                 double* w, double3 lenv) {
  const double len[3] = {lenv.x, lenv.y, lenv.z};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = p.id[q];
    if (x)
      for (int d = 0; d < ndim; ++d) {
        double v = p.x[d][q];
        if (v < 0.0) v += len[d];
        else if (v >= len[d]) v -= len[d];
        if (v >= len[d] || v < 0.0) v = 0.0;
        x[d * np + o] = v;
      }
    if (u)
      for (int c = 0; c < 3; ++c) u[c * np + o] = p.u[c][q];
    if (w) w[o] = p.w[q];
  }
}

__global__ void unpermute_gain_kernel(PartPtrs p, int64_t np, double* out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = p.id[q];
    out[o] = p.wl[q];
    out[np + o] = p.wd[q];
  }
}

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

size_t particle_smem_bytes(int ndim, size_t tsize, const PartTile& t, int M) {
  (void)M;
  // the window: tile + (g - 1) guard cells below and g above, per axis
  size_t W1 = t.t[0] + 2 * t.g[0] - 1, W2 = t.t[1] + 2 * t.g[1] - 1,
         W3 = ndim == 3 ? t.t[2] + 2 * t.g[2] - 1 : 1;
  // E^n and the time-centred B over the window in the field precision; the current
  // per node: two int32 fixed-point sums per component for an FP32 deposit (24
  // bytes), three for FP64 (36 bytes; for 8-byte fields both forms fit in it)
  const size_t jb = tsize == 8 ? 36 : 24;
  return W1 * W2 * W3 * (6 * tsize + jb);
}

cudaError_t launch_bin_count(const PartPtrs& p, const GridArgs& g, const PartTile& t,
                             const BinBufs& b, int64_t np, cudaStream_t st, int kill_col) {
  cudaError_t e = cudaMemsetAsync(b.count, 0, sizeof(int64_t) * (t.ntiles + 1), st);
  if (e != cudaSuccess) return e;
  if (np > 0) bin_count_kernel<<<grid_for(np), 256, 0, st>>>(p, g, t, b, np, kill_col);
  return cudaGetLastError();
}

cudaError_t launch_bin_scan(const BinBufs& b, int64_t ntiles, cudaStream_t st) {
  const int64_t m = bin_scan_chunks(ntiles);
  bin_chunk_sum_kernel<<<(unsigned)m, kScanT, 0, st>>>(b, ntiles);
  bin_part_scan_kernel<<<1, 1024, 0, st>>>(b, m);
  bin_chunk_out_kernel<<<(unsigned)m, kScanT, 0, st>>>(b, ntiles);
  return cudaGetLastError();
}

int64_t bin_scan_chunks(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_bin_scatter(const PartPtrs& src, const PartPtrs& dst, const GridArgs& g,
                               const BinBufs& b, int64_t np, cudaStream_t st) {
  if (np > 0) bin_scatter_kernel<<<grid_for(np), 256, 0, st>>>(src, dst, g.ndim, b, np);
  return cudaGetLastError();
}

cudaError_t launch_unpermute(const PartPtrs& p, int ndim, int64_t np, double* x, double* u,
                             double* w, const double* len, cudaStream_t st) {
  if (np > 0)
    unpermute_kernel<<<grid_for(np), 256, 0, st>>>(p, ndim, np, x, u, w,
                                                   make_double3(len[0], len[1], len[2]));
  return cudaGetLastError();
}

__global__ void mark_alive_kernel(const int64_t* id, int64_t kept, int64_t* flag) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < kept;
       q += (int64_t)gridDim.x * blockDim.x)
    flag[id[q]] = 1;
}

__global__ void renumber_kernel(int64_t* id, int64_t kept, const int64_t* rank) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < kept;
       q += (int64_t)gridDim.x * blockDim.x)
    id[q] = rank[id[q]];
}

cudaError_t launch_renumber(int64_t* id, int64_t np_old, int64_t kept, int64_t* tmp,
                            cudaStream_t st) {
  int64_t* flag = tmp;
  int64_t* rank = tmp + np_old;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int64_t) * np_old, st);
  if (e != cudaSuccess || kept == 0) return e;
  mark_alive_kernel<<<grid_for(kept), 256, 0, st>>>(id, kept, flag);
  BinBufs b{};
  b.count = flag;
  b.start = rank;
  b.part = tmp + 2 * np_old + 1;
  if ((e = launch_bin_scan(b, np_old, st)) != cudaSuccess) return e;
  renumber_kernel<<<grid_for(kept), 256, 0, st>>>(id, kept, rank);
  return cudaGetLastError();
}

cudaError_t launch_unpermute_gain(const PartPtrs& p, int64_t np, double* out, cudaStream_t st) {
  if (np > 0 && p.wl) unpermute_gain_kernel<<<grid_for(np), 256, 0, st>>>(p, np, out);
  return cudaGetLastError();
}

}  // namespace pic
