// batch.cu -- ensembles of independent 2D runs advanced by one persistent kernel.
//
// Every run keeps its own fields (in one pool), particles and step count.  One
// cooperative launch loops over the steps; in each step its CTAs take work
// items -- field tiles of any run (fused Faraday + Ampere, field_tile.cuh) and
// particle chunks of any run (gather/push/move/deposit from global memory,
// particle_core.cuh) -- and meet at a grid barrier before the next step.
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
#include "field_tile.cuh"
#include "laser_host.h"
#include "particle_core.cuh"

using namespace pic;

namespace {

struct RunInfo {
  int n1, n2;
  int64_t off;      // first cell of the run in each pool array
  int ntiles;       // field tiles of the run for the current tile shape
  int64_t p0, p1;   // particle range
  int64_t nsteps;   // steps of the current pic_batch_run
  int cur;          // parity of the buffers holding the run's state
};

template <typename T>
struct BatchArgs {
  RunInfo* runs;
  const int2* items;  // (run, sub): sub < ntiles -> field tile, else particle chunk
  int nitems;
  T* pool;            // [parity 0: E1 E2 E3 B1 B2 B3][parity 1: ...][J1 J2 J3], `total` cells each
  int64_t total;
  PartPtrs parts;
  StencilArgs<T> s;
  GridArgs gbase;     // dx, inv_dx, dx_dt, dt (sizes per run)
  PartArgs a;
  int TX, TY;
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

template <typename T>
__device__ void particle_chunk(const BatchArgs<T>& A, const StencilArgs<T>* sp, const RunInfo& R,
                               int chunk, int par) {
  const int64_t q = R.p0 + (int64_t)chunk * blockDim.x + threadIdx.x;
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
  for (int c = 0; c < 3; ++c) e[c] = pool_ptr(A, par * 6 + c, R.off);
  for (int c = 0; c < 3; ++c) {
    ve[c] = GlobView<T, true>{e[c], R.n1, R.n2, 1};
    vb[c] = BbarView<T, 2, true>{{e[0], e[1], e[2]}, pool_ptr(A, par * 6 + 3 + c, R.off), c,
                                 R.n1, R.n2, 1, sp};
    acc[c] = GlobAcc<T>{pool_ptr(A, 12 + c, R.off), R.n1, R.n2, 1};
  }
  int li[3] = {0, 0, 0};
  T fr[3] = {0, 0, 0};
  for (int d = 0; d < 2; ++d) {
    const double c = A.parts.x[d][q] * g.inv_dx[d];
    const double fl = floor(c);
    li[d] = (int)fl;
    fr[d] = (T)(c - fl);
  }
  advance_particle<T, 2>(ve, vb, acc, A.parts, q, li, fr, li, g, A.a, A.err);
}

template <typename T, int MT>
__global__ void __launch_bounds__(256, 3) batch_kernel(BatchArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ StencilArgs<T> s_sten;   // the particle path takes its address
  if (threadIdx.x == 0) s_sten = A.s;
  __syncthreads();
  unsigned epoch = 0;
  const int nphase = A.has_current ? 2 : 1;
  for (int64_t step = 0; step < A.max_steps; ++step) {
    for (int phase = 0; phase < nphase; ++phase) {
      for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
        const int2 w = A.items[it];
        const RunInfo R = A.runs[w.x];
        if (step >= R.nsteps) continue;
        const bool is_field = w.y < R.ntiles;
        if (A.has_current && ((phase == 1) != is_field)) continue;
        const int par = (R.cur + (int)step) & 1;
        if (is_field) {
          const T* e[3];
          const T* b[3];
          T* eo[3];
          T* bo[3];
          T* j[3];
          for (int c = 0; c < 3; ++c) {
            e[c] = pool_ptr(A, par * 6 + c, R.off);
            b[c] = pool_ptr(A, par * 6 + 3 + c, R.off);
            eo[c] = pool_ptr(A, (1 - par) * 6 + c, R.off);
            bo[c] = pool_ptr(A, (1 - par) * 6 + 3 + c, R.off);
            j[c] = pool_ptr(A, 12 + c, R.off);
          }
          field_tile<T, 2, true, MT>(e, b, A.has_current ? j : nullptr, eo, bo,
                                 FieldDims{R.n1, R.n2, 1}, A.s, (T)A.gbase.dt, A.TX, A.TY, 1,
                                 w.y, sm, A.has_current != 0);
          __syncthreads();  // the next item restages shared memory
        } else {
          particle_chunk<T>(A, &s_sten, R, w.y - R.ntiles, par);
        }
      }
      if (!grid_wait(A, epoch)) return;
    }
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
  int TX = 128, TY = 8;
  unsigned* bar = nullptr;
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

// work items for the current tile shape and particle set
pic_status build_items(pic_batch* b) {
  std::vector<int2> items;
  for (int r = 0; r < b->nruns; ++r) {
    RunInfo& R = b->runs[r];
    R.ntiles = ((R.n1 + b->TX - 1) / b->TX) * ((R.n2 + b->TY - 1) / b->TY);
    for (int t = 0; t < R.ntiles; ++t) items.push_back(make_int2(r, t));
  }
  for (int r = 0; r < b->nruns; ++r) {
    const RunInfo& R = b->runs[r];
    const int64_t n = R.p1 - R.p0;
    const int chunks = (int)((n + 255) / 256);
    for (int c = 0; c < chunks; ++c) items.push_back(make_int2(r, R.ntiles + c));
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
  A.TX = b->TX;
  A.TY = b->TY;
  A.max_steps = b->max_steps;
  A.has_current = b->has_current;
  A.bar = b->bar;
  A.err = b->err;
  A.timeout_ns = (long long)(b->timeout_s * 1e9);
  b->smem = field_tile_smem_elems(2, b->TX, b->TY, 1, b->M, (int)sizeof(T)) * sizeof(T);
  const BatchKernel<T> kern = batch_kernel_for<T>(b->M);
  BCK(b, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int nsm = 0, bps = 0;
  BCK(b, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
  BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, b->smem));
  if (bps < 1) return bfail(b, PIC_ERR_CUDA, "persistent kernel does not fit on an SM");
  b->bps = bps;
  b->grid = std::max(1, std::min(b->nitems, bps * nsm));
  A.expected = (unsigned)b->grid + (b->impossible ? 1u : 0u);

  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(256);
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
  return b->tsize == 8 ? launch_batch<double>(b) : launch_batch<float>(b);
}

}  // namespace

extern "C" {

pic_status pic_batch_init(const pic_batch_desc* d, double dt, const pic_coeffs* co, void* stream,
                          pic_batch** out) {
  if (!out) return PIC_ERR_ARG;
  *out = nullptr;
  if (!d || !co || d->nruns < 1 || !d->n1 || !d->n2 || !(dt > 0)) return PIC_ERR_ARG;
  if (d->precision != PIC_FP64 && d->precision != PIC_MIXED) return PIC_ERR_ARG;
  if (d->pusher != PIC_BORIS && d->pusher != PIC_ANALYTIC) return PIC_ERR_ARG;
  if (co->M < 1 || co->M > PIC_MAX_M || !co->cE || !co->cB) return PIC_ERR_ARG;
  if (!(d->dx[0] > 0) || !(d->dx[1] > 0)) return PIC_ERR_ARG;
  pic_batch* b = new pic_batch();
  b->nruns = d->nruns;
  b->precision = d->precision;
  b->pusher = d->pusher;
  b->tsize = d->precision == PIC_FP64 ? 8 : 4;
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
  int64_t off = 0;
  for (int r = 0; r < b->nruns; ++r) {
    if (d->n1[r] < 1 || d->n2[r] < 1) {
      delete b;
      return PIC_ERR_ARG;
    }
    RunInfo& R = b->runs[r];
    R = RunInfo{d->n1[r], d->n2[r], off, 0, 0, 0, 0, 0};
    // runs start on 256-byte boundaries in every pool array (vector accesses)
    off += ((int64_t)d->n1[r] * d->n2[r] + 63) / 64 * 64;
    b->cells += (int64_t)d->n1[r] * d->n2[r];
  }
  b->total = off;
  fill_stencil_b<double>(b, b->sd);
  fill_stencil_b<float>(b, b->sf);
  b->TX = b->tsize == 4 ? 256 : 128;
  b->TY = 8;
  auto init_fail = [&](pic_status s) {
    pic_batch_destroy(b);
    return s;
  };
  if (cudaMalloc(&b->pool, b->tsize * b->total * 15) != cudaSuccess) return init_fail(PIC_ERR_OOM);
  if (cudaMemsetAsync(b->pool, 0, b->tsize * b->total * 15, b->stream) != cudaSuccess ||
      cudaMalloc(&b->d_runs, sizeof(RunInfo) * b->nruns) != cudaSuccess ||
      cudaMalloc(&b->bar, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&b->err, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(b->err, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess)
    return init_fail(PIC_ERR_CUDA);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return init_fail(PIC_ERR_CUDA);
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
  cudaFree(b->d_runs);
  cudaFree(b->d_items);
  cudaFree(b->bar);
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
    GridArgs g{};
    g.ndim = 2;
    g.n[0] = R.n1;
    g.n[1] = R.n2;
    g.n[2] = 1;
    g.dx[0] = b->dx[0];
    g.dx[1] = b->dx[1];
    g.dx[2] = 1.0;
    g.ncell = (int64_t)R.n1 * R.n2;
    const int par = R.cur;
    if (e == cudaSuccess) {
      if (b->tsize == 8) {
        FieldPtrs<double> f;
        for (int c = 0; c < 3; ++c) {
          f.e[c] = (double*)b->pool + (int64_t)(par * 6 + c) * b->total + R.off;
          f.b[c] = (double*)b->pool + (int64_t)(par * 6 + 3 + c) * b->total + R.off;
          f.j[c] = nullptr;
        }
        e = launch_laser_expand<double>(f, g, dev, dev + R.n1, l.w0, l.x2c, l.x3c, b->stream);
      } else {
        FieldPtrs<float> f;
        for (int c = 0; c < 3; ++c) {
          f.e[c] = (float*)b->pool + (int64_t)(par * 6 + c) * b->total + R.off;
          f.b[c] = (float*)b->pool + (int64_t)(par * 6 + 3 + c) * b->total + R.off;
          f.j[c] = nullptr;
        }
        e = launch_laser_expand<float>(f, g, dev, dev + R.n1, l.w0, l.x2c, l.x3c, b->stream);
      }
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
  static const int cand32[][2] = {{64, 8}, {128, 4}, {128, 8}, {256, 4}, {256, 8}, {512, 4}};
  static const int cand64[][2] = {{64, 4}, {64, 8}, {128, 4}, {128, 8}, {256, 4}};
  const int (*cand)[2] = b->tsize == 4 ? cand32 : cand64;
  const int ncand = b->tsize == 4 ? 6 : 5;
  std::vector<int64_t> saved(b->nruns);
  for (int r = 0; r < b->nruns; ++r) {
    saved[r] = b->runs[r].nsteps;
    b->runs[r].nsteps = trial_steps;
  }
  float best = 1e30f;
  int bx = b->TX, by = b->TY;
  pic_status st = PIC_OK;
  for (int c = 0; c < ncand && st == PIC_OK; ++c) {
    b->TX = cand[c][0];
    b->TY = cand[c][1];
    if (field_tile_smem_elems(2, b->TX, b->TY, 1, b->M, (int)b->tsize) * b->tsize > 200 * 1024)
      continue;
    st = build_items(b);
    if (st == PIC_OK) st = run_now(b);
    if (st == PIC_OK && b->last_ms < best) {
      best = b->last_ms;
      bx = b->TX;
      by = b->TY;
    }
  }
  b->TX = bx;
  b->TY = by;
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
  const char* src = (const char*)b->pool + ((int64_t)slot * b->total + R.off) * b->tsize;
  if (b->tsize == 8) {
    BCK(b, cudaMemcpy(buf, src, sizeof(double) * n, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(n);
    BCK(b, cudaMemcpy(tmp.data(), src, sizeof(float) * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) buf[i] = tmp[i];
  }
  return PIC_OK;
}

pic_status pic_batch_get_info(pic_batch* b, pic_batch_info* info) {
  if (!b || !info) return bfail(b, PIC_ERR_ARG, "null argument");
  memset(info, 0, sizeof *info);
  info->tile[0] = b->TX;
  info->tile[1] = b->TY;
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
  return PIC_OK;
}

pic_status pic_batch_set_barrier(pic_batch* b, double timeout_s, int impossible) {
  if (!b || !(timeout_s > 0)) return bfail(b, PIC_ERR_ARG, "timeout must be positive");
  b->timeout_s = timeout_s;
  b->impossible = impossible ? 1 : 0;
  b->graph_dirty = true;
  return PIC_OK;
}

}  // extern "C"
