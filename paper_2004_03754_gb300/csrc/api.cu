// api.cu -- host side of libpic: context, validation, setup, step orchestration.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.cuh"
#include "field_tile.cuh"
#include "correction_host.h"
#include "laser_host.h"

using namespace pic;

static std::string g_init_error;

namespace {

const char* cuda_msg(cudaError_t e) { return cudaGetErrorString(e); }

#define CK(ctx, call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      (ctx)->err = std::string(#call) + ": " + cuda_msg(e_);                           \
      return e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA;             \
    }                                                                                  \
  } while (0)

pic_status fail(pic_ctx* c, pic_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

double kspace(int M, const double* c, double k, double dx) {
  double s = 0;
  for (int j = 1; j <= M; ++j) s += c[j - 1] * sin((2 * j - 1) * k * dx / 2.0);
  return s / (dx / 2.0);
}

template <typename T>
FieldPtrs<T> fields(pic_ctx* c, int set) {
  FieldPtrs<T> f;
  for (int k = 0; k < 3; ++k) {
    f.e[k] = (T*)c->fe[set][k];
    f.b[k] = (T*)c->fb[set][k];
    f.j[k] = (T*)c->fj[k];
  }
  return f;
}

void* comp_ptr(pic_ctx* c, int comp) {
  if (comp < 3) return c->fe[c->cur][comp];
  if (comp < 6) return c->fb[c->cur][comp - 3];
  return c->fj[comp - 6];
}

// particle tile and guard: guard = 3 + drift allowance; rebin interval chosen so
// that no particle (|v| < c) can leave its window between rebinnings.
void choose_particle_tiles(pic_ctx* c) {
  const int nd = c->grid.ndim;
  PartTile& t = c->ptile;
  int tgt[3], K = 8;
  if (nd == 2) {
    tgt[0] = 32; tgt[1] = 16; tgt[2] = 1;
  } else {
    // 3D (few particles per tile): re-binning every step keeps the guard at 3
    // cells above and 2 below, so the staged windows (13x13x9 nodes, 73 KB in
    // FP32 with the fixed-point current) fit 3 CTAs per SM; a sweep on the
    // 512x128x128 case found this faster than larger tiles or guards
    tgt[0] = 8; tgt[1] = 8; tgt[2] = 4;
    K = 1;
  }
  for (;;) {
    for (int d = 0; d < 3; ++d) {
      if (d < nd) {
        t.t[d] = std::min(tgt[d], c->g.n[d]);
        const double cfl = c->dt * c->g.inv_dx[d];
        t.g[d] = 3 + (int)ceil(cfl * (K - 1) - 1e-12);
      } else {
        t.t[d] = 1;
        t.g[d] = 0;
      }
    }
    if (particle_smem_bytes(nd, c->tsize, t, c->M) <= 200 * 1024 || K == 1) break;
    --K;
  }
  int Kmax = 1 << 20;
  for (int d = 0; d < nd; ++d) {
    const double cfl = c->dt * c->g.inv_dx[d];
    if (cfl > 0) Kmax = std::min(Kmax, 1 + (int)floor((t.g[d] - 3) / cfl + 1e-12));
  }
  c->sort_interval = std::max(1, Kmax);
  t.ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    t.nt[d] = d < nd ? (c->g.n[d] + t.t[d] - 1) / t.t[d] : 1;
    t.ntiles *= t.nt[d];
  }
}

template <typename T>
void fill_stencil(pic_ctx* c, StencilArgs<T>& s) {
  s.M = c->M;
  for (int j = 0; j < PIC_MAX_M; ++j) {
    s.kE[j] = (T)(j < c->M ? c->dt * c->cE[j] / c->g.dx[0] : 0.0);
    s.kB[j] = (T)(j < c->M ? c->dt * c->cB[j] / c->g.dx[0] : 0.0);
  }
  s.y2 = (T)(c->dt / c->g.dx[1]);
  s.y3 = (T)(c->grid.ndim == 3 ? c->dt / c->g.dx[2] : 0.0);
}

// Taps of the x1 current correction on this grid's rows (correction_host.h),
// stored in the field precision.
pic_status build_correction(pic_ctx* c) {
  std::vector<double> taps;
  if (!inv_circulant_taps(c->g.n[0], c->g.dx[0], c->M, c->cB, taps, c->taps_lo))
    return fail(c, PIC_ERR_ARG, "C^B gives [k]_B1 = 0 at a grid mode");
  c->taps_n = (int)taps.size();
  if (c->grid.precision == PIC_FP64) {
    CK(c, cudaMalloc(&c->taps, sizeof(double) * taps.size()));
    CK(c, cudaMemcpy(c->taps, taps.data(), sizeof(double) * taps.size(), cudaMemcpyHostToDevice));
  } else if (c->grid.precision == PIC_COMPENSATED) {
    std::vector<pic::dfl> td;
    for (double v : taps) td.push_back(pic::dfl(v));
    CK(c, cudaMalloc(&c->taps, sizeof(pic::dfl) * td.size()));
    CK(c, cudaMemcpy(c->taps, td.data(), sizeof(pic::dfl) * td.size(), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> tf(taps.begin(), taps.end());
    CK(c, cudaMalloc(&c->taps, sizeof(float) * tf.size()));
    CK(c, cudaMemcpy(c->taps, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice));
  }
  return PIC_OK;
}

pic_status alloc_particles(pic_ctx* c, int64_t n) {
  if (n <= c->cap) return PIC_OK;
  for (int s = 0; s < 2; ++s) {
    PartPtrs& p = c->parts[s];
    for (int d = 0; d < 3; ++d) {
      cudaFree(p.x[d]);
      cudaFree(p.u[d]);
      p.x[d] = p.u[d] = nullptr;
    }
    cudaFree(p.w);
    cudaFree(p.id);
    cudaFree(p.wl);
    cudaFree(p.wd);
    p.w = nullptr;
    p.id = nullptr;
    p.wl = p.wd = nullptr;
  }
  cudaFree(c->bins.key);
  cudaFree(c->bins.slot);
  cudaFree(c->bins.strag);
  c->bins.key = c->bins.slot = nullptr;
  c->bins.strag = nullptr;
  c->cap = 0;
  for (int s = 0; s < 2; ++s) {
    PartPtrs& p = c->parts[s];
    for (int d = 0; d < c->grid.ndim; ++d) CK(c, cudaMalloc(&p.x[d], sizeof(double) * n));
    for (int d = 0; d < 3; ++d) CK(c, cudaMalloc(&p.u[d], sizeof(double) * n));
    CK(c, cudaMalloc(&p.w, sizeof(double) * n));
    CK(c, cudaMalloc(&p.id, sizeof(int64_t) * n));
    if (c->gain) {
      CK(c, cudaMalloc(&p.wl, sizeof(double) * n));
      CK(c, cudaMalloc(&p.wd, sizeof(double) * n));
    }
  }
  CK(c, cudaMalloc(&c->bins.key, sizeof(int) * n));
  CK(c, cudaMalloc(&c->bins.slot, sizeof(int) * n));
  CK(c, cudaMalloc(&c->bins.strag, sizeof(int64_t) * n));
  c->cap = n;
  return PIC_OK;
}

cudaEvent_t take_event(pic_ctx* c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII pair of events around one kernel group (group ids: 0 rebin, 1 particles,
// 2 stragglers, 3 correction, 4 fields); no-op unless timing is enabled.
struct TimedScope {
  pic_ctx* c;
  int group;
  cudaEvent_t a = nullptr;
  TimedScope(pic_ctx* ctx, int g, int nlaunch) : c(ctx), group(g) {
    if (!c->timing) return;
    a = take_event(c);
    cudaEventRecord(a, c->stream);
    c->t_launches += nlaunch;
  }
  ~TimedScope() {
    if (!c->timing) return;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, c->stream);
    c->tev.push_back({group, {a, b}});
  }
};

pic_status rebin(pic_ctx* c) {
  if (c->np == 0) {
    c->steps_since_sort = 0;
    return PIC_OK;
  }
  PartPtrs& src = c->parts[c->pcur];
  PartPtrs& dst = c->parts[1 - c->pcur];
  TimedScope ts(c, 0, 3);
  CK(c, launch_bin_count(src, c->g, c->ptile, c->bins, c->np, c->stream));
  CK(c, launch_bin_scan(c->bins, c->ptile.ntiles, c->stream));
  CK(c, launch_bin_scatter(src, dst, c->g, c->bins, c->np, c->stream));
  c->pcur = 1 - c->pcur;
  c->steps_since_sort = 0;
  return PIC_OK;
}

template <typename T>
pic_status one_step(pic_ctx* c, const StencilArgs<T>& s) {
  if (c->steps_since_sort >= c->sort_interval) {
    pic_status st = rebin(c);
    if (st != PIC_OK) return st;
  }
  for (int k = 0; k < 3; ++k) CK(c, cudaMemsetAsync(c->fj[k], 0, c->tsize * c->g.ncell, c->stream));
  FieldPtrs<T> f = fields<T>(c, c->cur);
  if (c->np > 0) {
    CK(c, cudaMemsetAsync(c->bins.strag_count, 0, sizeof(unsigned long long), c->stream));
    PartArgs a{c->qm, c->grid.pusher, c->np};
    {
      TimedScope ts(c, 1, c->grid.ndim == 3 ? 2 : 1);
      BbarPtrs<T> bg{{(T*)c->bbar[0], (T*)c->bbar[1], (T*)c->bbar[2]}};
      CK(c, launch_particle_step<T>(f, bg, c->parts[c->pcur], c->g, s, c->ptile, a, c->bins,
                                    c->stream));
    }
    {
      TimedScope ts(c, 2, 1);
      BbarPtrs<T> bg{{(T*)c->bbar[0], (T*)c->bbar[1], (T*)c->bbar[2]}};
      CK(c, launch_straggler_step<T>(f, bg, c->parts[c->pcur], c->g, s, a, c->bins, c->np,
                                     c->stream));
    }
  }
  if (c->corr) {
    TimedScope ts(c, 3, 1);
    CK(c, launch_correct_j1<T>((T*)c->fj[0], (T*)c->jtmp, c->g, (const T*)c->taps, c->taps_lo,
                               c->taps_n, c->corr_path, c->stream));
  }
  FieldPtrs<T> o = fields<T>(c, 1 - c->cur);
  {
    TimedScope ts(c, 4, 1);
    CK(c, launch_field_step<T>(f, o, c->g, s, c->ftile, c->bins.err, c->stream));
  }
  if (c->timing) c->t_steps++;
  c->cur = 1 - c->cur;
  c->steps_since_sort++;
  c->steps_done++;
  return PIC_OK;
}

pic_status ensure_scratch(pic_ctx* c) {
  if (!c->scratch) CK(c, cudaMalloc(&c->scratch, sizeof(double) * c->g.ncell));
  return PIC_OK;
}

pic_status check_err_word(pic_ctx* c) {
  unsigned h = 0;
  CK(c, cudaMemcpyAsync(&h, c->bins.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (h) {
    std::string m = "device check failed:";
    if (h & ERRBIT_MOVE) m += " particle moved >= 1 cell in a step;";
    if (h & ERRBIT_ANALYTIC) m += " analytic pusher proper-time iteration did not converge;";
    if (h & ERRBIT_NONFINITE) m += " non-finite particle state;";
    if (h & ERRBIT_POSITION) m += " particle position outside the box at load;";
    if (h & ERRBIT_TIMEOUT) m += " field staging copy wait timed out;";
    c->err = m;
    CK(c, cudaMemsetAsync(c->bins.err, 0, sizeof(unsigned), c->stream));
    return PIC_ERR_DEVICE_CHECK;
  }
  return PIC_OK;
}

__global__ void check_positions_kernel(PartPtrs p, GridArgs g, int64_t np, unsigned* err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
       q += (int64_t)gridDim.x * blockDim.x) {
    p.id[q] = q;
    for (int d = 0; d < g.ndim; ++d) {
      const double x = p.x[d][q];
      if (!(x >= 0.0 && x < g.len[d])) atomicOr(err, 8u);
    }
  }
}

}  // namespace

// Checkpoint layout (pic_save_state / pic_load_state): a header, then E1 E2 E3
// B1 B2 B3 (n1*n2*n3 values each, field precision, x1 fastest), then the
// particles in load order as FP64 arrays x (ndim*np), u (3*np), w (np).
struct StateHeader {
  char magic[8];
  int32_t version, ndim, precision, M;
  int32_t n[3], pad;
  double dx[3], dt, qm;
  double cE[PIC_MAX_M], cB[PIC_MAX_M];
  int64_t np, steps_done;
  uint64_t field_bytes, part_bytes;
};
constexpr char kStateMagic[8] = {'P', 'I', 'C', 'S', 'T', 'A', 'T', 'E'};
constexpr size_t kStateHdr = (sizeof(StateHeader) + 63) / 64 * 64;

size_t state_bytes(const pic_ctx* c) {
  return kStateHdr + 6 * (size_t)c->g.ncell * c->tsize +
         (size_t)c->np * (size_t)(c->grid.ndim + 4) * sizeof(double);
}

extern "C" {

pic_status pic_init(const pic_grid* grid, double dt, const pic_coeffs* coeffs, void* stream,
                    pic_ctx** out) {
  if (!out) return PIC_ERR_ARG;
  *out = nullptr;
  g_init_error.clear();
  auto bad = [&](const char* m) {
    g_init_error = m;
    return PIC_ERR_ARG;
  };
  if (!grid || !coeffs) return bad("null grid or coefficients");
  if (grid->ndim != 2 && grid->ndim != 3) return bad("ndim must be 2 or 3");
  if (grid->precision != PIC_FP64 && grid->precision != PIC_MIXED &&
      grid->precision != PIC_COMPENSATED)
    return bad("bad precision");
  if (grid->pusher != PIC_BORIS && grid->pusher != PIC_ANALYTIC && grid->pusher != PIC_HC)
    return bad("bad pusher");
  if (grid->shape != 0 && grid->shape != PIC_SHAPE_QUADRATIC)
    return bad("shape: only the quadratic B-spline (App. A) is built");
  if (grid->boundary != 0 && grid->boundary != PIC_BOUNDARY_PERIODIC)
    return bad("boundary: only periodic boundaries are built");
  if (coeffs->M < 1 || coeffs->M > PIC_MAX_M || !coeffs->cE || !coeffs->cB)
    return bad("M out of range or null coefficient array");
  if (!(dt > 0) || !isfinite(dt)) return bad("dt must be positive");
  int64_t ncell = 1;
  for (int d = 0; d < grid->ndim; ++d) {
    if (grid->n[d] < 1 || !(grid->dx[d] > 0) || !isfinite(grid->dx[d])) return bad("bad n or dx");
    ncell *= grid->n[d];
  }
  if (ncell > ((int64_t)1 << 40)) return bad("grid too large");
  pic_ctx* c = new pic_ctx();
  c->grid = *grid;
  if (grid->ndim == 2) {
    c->grid.n[2] = 1;
    c->grid.dx[2] = 1.0;
  }
  c->dt = dt;
  c->M = coeffs->M;
  for (int j = 0; j < c->M; ++j) {
    c->cE[j] = coeffs->cE[j];
    c->cB[j] = coeffs->cB[j];
    if (!isfinite(c->cE[j]) || !isfinite(c->cB[j])) {
      delete c;
      return bad("non-finite coefficient");
    }
  }
  c->stream = (cudaStream_t)stream;
  c->tsize = grid->precision == PIC_MIXED ? sizeof(float) : 8;  // FP64 or an FP32 pair
  GridArgs& g = c->g;
  g.ndim = grid->ndim;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = c->grid.n[d];
    g.dx[d] = c->grid.dx[d];
    g.inv_dx[d] = 1.0 / g.dx[d];
    g.len[d] = g.n[d] * g.dx[d];
    g.dx_dt[d] = g.dx[d] / dt;
  }
  g.dt = dt;
  g.ncell = ncell;
  // exact CFL condition, Eq. (21), on a fine k1 grid; x2/x3 Yee terms at Nyquist
  {
    const int nk = 20001;
    double pmax = 0, pmin = 0;
    for (int q = 0; q < nk; ++q) {
      const double k = M_PI / g.dx[0] * q / (nk - 1);
      const double p = kspace(c->M, c->cB, k, g.dx[0]) * kspace(c->M, c->cE, k, g.dx[0]);
      pmax = std::max(pmax, p);
      pmin = std::min(pmin, p);
    }
    double yee = 0, suff = 0, sB = 0, sE = 0;
    for (int d = 1; d < grid->ndim; ++d) {
      yee += (2.0 / g.dx[d]) * (2.0 / g.dx[d]);
      suff += 1.0 / (g.dx[d] * g.dx[d]);
    }
    for (int j = 0; j < c->M; ++j) {
      sB += fabs(c->cB[j]);
      sE += fabs(c->cE[j]);
    }
    c->cfl_lhs = (dt / 2) * (dt / 2) * (pmax + yee);
    c->cfl_suff = 1.0 / sqrt(sB * sE / (g.dx[0] * g.dx[0]) + suff);
    if (c->cfl_lhs > 1.0 + 1e-12 || pmin < -1e-12 * std::max(pmax, 1e-300)) {
      char buf[160];
      snprintf(buf, sizeof buf, "CFL violated: max (dt/2)^2 ([k]_B[k]_E + Yee) = %.6g, min [k]_B[k]_E = %.3g",
               c->cfl_lhs, pmin);
      g_init_error = buf;
      delete c;
      return PIC_ERR_CFL;
    }
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    g_init_error = "no CUDA device";
    delete c;
    return PIC_ERR_CUDA;
  }
  fill_stencil<double>(c, c->sd);
  fill_stencil<float>(c, c->sf);
  fill_stencil<pic::dfl>(c, c->sdf);
  c->corr = false;
  for (int j = 0; j < c->M; ++j)
    if (c->cB[j] != (j == 0 ? 1.0 : 0.0)) c->corr = true;
  // field tiles: wide along x1 to amortise the 2M-1 halo of the x1 stencils
  // (shapes from a sweep on the 4096x1024 and 512x128x128 grids)
  c->ftile.threads = 256;
  c->ftile.staging = 0;
  // 2D rows (J read into registers, not staged): FP32 224 columns x 4 warps x 3
  // stages, 0.0539 ms at 4096x1024 against 0.0600 ms for 352 x 2 x 3
  c->ftile.sw = 224;
  c->ftile.rows = 0;
  c->ftile.warps = c->tsize == 4 ? 4 : 2;
  c->ftile.stages = c->tsize == 4 ? 3 : 2;
  if (grid->ndim == 2) {
    c->ftile.t[0] = c->tsize == 4 ? 256 : 128; c->ftile.t[1] = c->tsize == 4 ? 4 : 8;
    c->ftile.t[2] = 1;
  } else {
    c->ftile.t[0] = c->tsize == 4 ? 128 : 64; c->ftile.t[1] = 4; c->ftile.t[2] = 2;
    // rows streamed along x2 by CTAs of P warps over P consecutive x3 planes, two
    // stages: at 1024x256x256, FP32 fields 128-column strips, P = 4 (1.09 ms
    // against 2.07 ms for one warp per plane and 5.4 ms on the CTA tiles);
    // compensated pairs 64 columns, P = 8 (7.6 ms against 14.2 ms); FP64 64
    // columns, P = 4 (29.4 ms against 37.6 ms on the CTA tiles)
    c->ftile.sw = grid->precision == PIC_MIXED ? 128 : 64;
    c->ftile.stages = 2;
    c->ftile.warps = grid->precision == PIC_COMPENSATED ? 8 : 4;
  }
  choose_particle_tiles(c);
  auto init_fail = [&](pic_status s) {
    g_init_error = c->err;
    pic_destroy(c);
    return s;
  };
  const size_t bytes = c->tsize * ncell;
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      if (cudaMalloc(&c->fe[s][k], bytes) != cudaSuccess || cudaMalloc(&c->fb[s][k], bytes) != cudaSuccess) {
        c->err = "field allocation failed";
        return init_fail(PIC_ERR_OOM);
      }
      cudaMemsetAsync(c->fe[s][k], 0, bytes, c->stream);
      cudaMemsetAsync(c->fb[s][k], 0, bytes, c->stream);
    }
  for (int k = 0; k < 3; ++k) {
    if (cudaMalloc(&c->fj[k], bytes) != cudaSuccess) {
      c->err = "field allocation failed";
      return init_fail(PIC_ERR_OOM);
    }
    cudaMemsetAsync(c->fj[k], 0, bytes, c->stream);
  }
  // the time-centred B of each step (read by the particle tiles)
  for (int k = 0; k < 3; ++k)
    if (cudaMalloc(&c->bbar[k], bytes) != cudaSuccess) {
      c->err = "field allocation failed";
      return init_fail(PIC_ERR_OOM);
    }
  if (c->corr) {
    if (cudaMalloc(&c->jtmp, bytes) != cudaSuccess) {
      c->err = "allocation failed";
      return init_fail(PIC_ERR_OOM);
    }
    pic_status st = build_correction(c);
    if (st != PIC_OK) return init_fail(st);
  }
  c->bins_ntiles = c->ptile.ntiles;
  if (cudaMalloc(&c->bins.count, sizeof(int64_t) * (c->ptile.ntiles + 1)) != cudaSuccess ||
      cudaMalloc(&c->bins.start, sizeof(int64_t) * (c->ptile.ntiles + 2)) != cudaSuccess ||
      cudaMalloc(&c->bins.part, sizeof(int64_t) * bin_scan_chunks(c->ptile.ntiles + 1)) !=
          cudaSuccess ||
      cudaMalloc(&c->bins.strag_count, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&c->bins.err, sizeof(unsigned)) != cudaSuccess) {
    c->err = "allocation failed";
    return init_fail(PIC_ERR_OOM);
  }
  cudaMemsetAsync(c->bins.err, 0, sizeof(unsigned), c->stream);
  cudaMemsetAsync(c->bins.start, 0, sizeof(int64_t) * (c->ptile.ntiles + 2), c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    c->err = cuda_msg(e);
    return init_fail(PIC_ERR_CUDA);
  }
  *out = c;
  return PIC_OK;
}

pic_status pic_destroy(pic_ctx* c) {
  if (!c) return PIC_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      cudaFree(c->fe[s][k]);
      cudaFree(c->fb[s][k]);
    }
  for (int k = 0; k < 3; ++k) {
    cudaFree(c->fj[k]);
    cudaFree(c->bbar[k]);
  }
  cudaFree(c->jtmp);
  cudaFree(c->scratch);
  cudaFree(c->rbuf);
  for (auto& g : c->sgraph)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  cudaFree(c->taps);
  for (int s = 0; s < 2; ++s) {
    for (int d = 0; d < 3; ++d) {
      cudaFree(c->parts[s].x[d]);
      cudaFree(c->parts[s].u[d]);
    }
    cudaFree(c->parts[s].w);
    cudaFree(c->parts[s].id);
    cudaFree(c->parts[s].wl);
    cudaFree(c->parts[s].wd);
  }
  cudaFree(c->bins.count);
  cudaFree(c->bins.start);
  cudaFree(c->bins.part);
  cudaFree(c->mw_tmp);
  spectral_free(c->spec);
  cudaFree(c->bins.key);
  cudaFree(c->bins.slot);
  cudaFree(c->bins.strag);
  cudaFree(c->bins.strag_count);
  cudaFree(c->bins.err);
  for (auto& t : c->tev) {
    cudaEventDestroy(t.second.first);
    cudaEventDestroy(t.second.second);
  }
  for (auto e : c->evpool) cudaEventDestroy(e);
  delete c;
  return PIC_OK;
}

const char* pic_last_error(const pic_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

pic_status pic_load_field(pic_ctx* c, int comp, const double* buf, int on_device) {
  if (!c || !buf || comp < 0 || comp > 5) return fail(c, PIC_ERR_ARG, "bad component or buffer");
  CK(c, cudaSetDevice(c->device));
  const double* src = buf;
  if (!on_device) {
    pic_status st = ensure_scratch(c);
    if (st != PIC_OK) return st;
    CK(c, cudaMemcpyAsync(c->scratch, buf, sizeof(double) * c->g.ncell, cudaMemcpyHostToDevice,
                          c->stream));
    src = c->scratch;
  }
  void* dst = comp_ptr(c, comp);
  if (c->grid.precision == PIC_FP64)
    CK(c, cudaMemcpyAsync(dst, src, sizeof(double) * c->g.ncell, cudaMemcpyDeviceToDevice, c->stream));
  else if (c->grid.precision == PIC_COMPENSATED)
    CK(c, launch_convert_in<pic::dfl>((pic::dfl*)dst, src, c->g.ncell, c->stream));
  else
    CK(c, launch_convert_in<float>((float*)dst, src, c->g.ncell, c->stream));
  if (!on_device) CK(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_read_field(pic_ctx* c, int comp, double* buf, int on_device) {
  if (!c || !buf || comp < 0 || comp > PIC_BBAR3) return fail(c, PIC_ERR_ARG, "bad component or buffer");
  CK(c, cudaSetDevice(c->device));
  double* dst = buf;
  if (!on_device) {
    pic_status st = ensure_scratch(c);
    if (st != PIC_OK) return st;
    dst = c->scratch;
  }
  if (comp >= PIC_BBAR1) {
    if (c->grid.precision == PIC_FP64)
      CK(c, launch_bbar<double>(fields<double>(c, c->cur), c->g, c->sd, dst, comp - PIC_BBAR1, c->stream));
    else if (c->grid.precision == PIC_COMPENSATED)
      CK(c, launch_bbar<pic::dfl>(fields<pic::dfl>(c, c->cur), c->g, c->sdf, dst, comp - PIC_BBAR1,
                                  c->stream));
    else
      CK(c, launch_bbar<float>(fields<float>(c, c->cur), c->g, c->sf, dst, comp - PIC_BBAR1, c->stream));
  } else if (c->grid.precision == PIC_FP64) {
    CK(c, cudaMemcpyAsync(dst, comp_ptr(c, comp), sizeof(double) * c->g.ncell,
                          cudaMemcpyDeviceToDevice, c->stream));
  } else if (c->grid.precision == PIC_COMPENSATED) {
    CK(c, launch_convert_out<pic::dfl>(dst, (const pic::dfl*)comp_ptr(c, comp), c->g.ncell, c->stream));
  } else {
    CK(c, launch_convert_out<float>(dst, (const float*)comp_ptr(c, comp), c->g.ncell, c->stream));
  }
  if (!on_device) {
    CK(c, cudaMemcpyAsync(buf, dst, sizeof(double) * c->g.ncell, cudaMemcpyDeviceToHost, c->stream));
    return check_err_word(c);
  }
  return PIC_OK;
}

pic_status pic_load_laser(pic_ctx* c, const pic_laser* L) {
  if (!c || !L) return fail(c, PIC_ERR_ARG, "null argument");
  if (!(L->L_env > 0) || L->L_env > c->g.len[0] || !isfinite(L->a0) || !(L->k0 > 0))
    return fail(c, PIC_ERR_ARG, "laser envelope must fit the box, k0 > 0, finite a0");
  CK(c, cudaSetDevice(c->device));
  const int n = c->g.n[0];
  std::vector<double> ep(n), bp(n);
  laser_profiles(n, c->g.dx[0], c->dt, c->M, c->cE, c->cB, *L, ep.data(), bp.data());
  double* dev = nullptr;
  CK(c, cudaMalloc(&dev, sizeof(double) * 2 * n));
  cudaError_t e = cudaMemcpyAsync(dev, ep.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dev + n, bp.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    if (c->grid.precision == PIC_FP64)
      e = launch_laser_expand<double>(fields<double>(c, c->cur), c->g, dev, dev + n, L->w0, L->x2c,
                                      L->x3c, c->stream);
    else if (c->grid.precision == PIC_COMPENSATED)
      e = launch_laser_expand<pic::dfl>(fields<pic::dfl>(c, c->cur), c->g, dev, dev + n, L->w0,
                                        L->x2c, L->x3c, c->stream);
    else
      e = launch_laser_expand<float>(fields<float>(c, c->cur), c->g, dev, dev + n, L->w0, L->x2c,
                                     L->x3c, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dev);
  CK(c, e);
  return PIC_OK;
}

pic_status pic_load_particles(pic_ctx* c, int64_t n, const double* x, const double* u,
                              const double* w, double qm, int on_device) {
  if (!c || n < 0 || (n > 0 && (!x || !u || !w)) || !isfinite(qm))
    return fail(c, PIC_ERR_ARG, "bad particle arguments");
  if (n > (int64_t)INT32_MAX * 64) return fail(c, PIC_ERR_ARG, "too many particles");
  CK(c, cudaSetDevice(c->device));
  const int nd = c->grid.ndim;
  pic_status st = alloc_particles(c, n);
  if (st != PIC_OK) return st;
  ++c->epoch;  // particle buffers and count change: captured step graphs are stale
  c->np = n;
  c->qm = qm;
  c->pcur = 0;
  PartPtrs& p = c->parts[0];
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n > 0) {
    for (int d = 0; d < nd; ++d) CK(c, cudaMemcpyAsync(p.x[d], x + d * n, sizeof(double) * n, kind, c->stream));
    for (int d = 0; d < 3; ++d) CK(c, cudaMemcpyAsync(p.u[d], u + d * n, sizeof(double) * n, kind, c->stream));
    CK(c, cudaMemcpyAsync(p.w, w, sizeof(double) * n, kind, c->stream));
    if (p.wl) {   // the energy-gain integrals start from zero with every load
      CK(c, cudaMemsetAsync(p.wl, 0, sizeof(double) * n, c->stream));
      CK(c, cudaMemsetAsync(p.wd, 0, sizeof(double) * n, c->stream));
    }
    int nb = (int)std::min<int64_t>((n + 255) / 256, 152 * 32);
    check_positions_kernel<<<nb, 256, 0, c->stream>>>(p, c->g, n, c->bins.err);
    CK(c, cudaGetLastError());
  }
  st = rebin(c);
  if (st != PIC_OK) return st;
  if (!on_device) {
    // the positions were checked on the device (check_positions_kernel)
    unsigned h = 0;
    CK(c, cudaMemcpyAsync(&h, c->bins.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (h & ERRBIT_POSITION) {
      CK(c, cudaMemsetAsync(c->bins.err, 0, sizeof(unsigned), c->stream));
      c->np = 0;
      return fail(c, PIC_ERR_ARG, "particle position outside [0, n*dx)");
    }
  }
  return PIC_OK;
}

// One step with the spectral x1 field path (FP64): Faraday first (forming
// B^{n+1/2} and the time-centred B), the particles reading that B, the current
// corrected along x1 in Fourier space, then Ampere.
pic_status one_step_spectral(pic_ctx* c) {
  if (c->steps_since_sort >= c->sort_interval) {
    pic_status st = rebin(c);
    if (st != PIC_OK) return st;
  }
  for (int k = 0; k < 3; ++k) CK(c, cudaMemsetAsync(c->fj[k], 0, c->tsize * c->g.ncell, c->stream));
  FieldPtrs<double> f = fields<double>(c, c->cur);
  FieldPtrs<double> o = fields<double>(c, 1 - c->cur);
  double* bb[3] = {(double*)c->bbar[0], (double*)c->bbar[1], (double*)c->bbar[2]};
  {
    TimedScope ts(c, 4, 5);
    CK(c, spectral_faraday(c, f, o.b, bb));
  }
  if (c->np > 0) {
    CK(c, cudaMemsetAsync(c->bins.strag_count, 0, sizeof(unsigned long long), c->stream));
    PartArgs a{c->qm, c->grid.pusher, c->np};
    a.bbar_ready = 1;
    BbarPtrs<double> bg{{bb[0], bb[1], bb[2]}};
    {
      TimedScope ts(c, 1, 1);
      CK(c, launch_particle_step<double>(f, bg, c->parts[c->pcur], c->g, c->sd, c->ptile, a,
                                         c->bins, c->stream));
    }
    {
      TimedScope ts(c, 2, 1);
      CK(c, launch_straggler_step<double>(f, bg, c->parts[c->pcur], c->g, c->sd, a, c->bins, c->np,
                                          c->stream));
    }
    TimedScope ts(c, 3, 3);
    CK(c, spectral_correct_j1(c, f.j[0]));
  }
  {
    TimedScope ts(c, 4, 5);
    CK(c, spectral_ampere(c, f, o.b, o.e));
  }
  if (c->timing) c->t_steps++;
  c->cur = 1 - c->cur;
  c->steps_since_sort++;
  c->steps_done++;
  return PIC_OK;
}

pic_status step_once(pic_ctx* c) {
  if (c->spec) return one_step_spectral(c);
  if (c->grid.precision == PIC_FP64) return one_step<double>(c, c->sd);
  if (c->grid.precision == PIC_COMPENSATED) return one_step<pic::dfl>(c, c->sdf);
  return one_step<float>(c, c->sf);
}

// One shift of the moving window (Sec. 4.1, reading of its boundary): the
// trailing x1 column mw_origin becomes fresh vacuum -- E, B and J cleared there --
// and the particles whose cell is that column leave: they are binned past the
// last tile by a re-binning and dropped, the kept ones renumbered in load order.
// The column is then the window's leading one.  No field data moves.
pic_status window_shift(pic_ctx* c) {
  const int64_t col = c->mw_origin;
  const size_t ts = c->tsize, pitch = ts * (size_t)c->g.n[0];
  const size_t rows = (size_t)(c->g.ncell / c->g.n[0]);
  for (int k = 0; k < 3; ++k) {
    void* arrs[3] = {c->fe[c->cur][k], c->fb[c->cur][k], c->fj[k]};
    for (void* a : arrs)
      CK(c, cudaMemset2DAsync((char*)a + col * ts, pitch, 0, ts, rows, c->stream));
  }
  if (c->np > 0) {
    PartPtrs& src = c->parts[c->pcur];
    PartPtrs& dst = c->parts[1 - c->pcur];
    const int64_t nt = c->ptile.ntiles;
    CK(c, launch_bin_count(src, c->g, c->ptile, c->bins, c->np, c->stream, (int)col));
    CK(c, launch_bin_scan(c->bins, nt + 1, c->stream));
    CK(c, launch_bin_scatter(src, dst, c->g, c->bins, c->np, c->stream));
    int64_t kept = 0;
    CK(c, cudaMemcpyAsync(&kept, c->bins.start + nt, sizeof(int64_t), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (kept < c->np) {
      // flags, ranks (np + 1) and the scan's chunk sums
      const int64_t need = 2 * c->np + 1 + bin_scan_chunks(c->np);
      if (c->mw_tmp_n < need) {
        cudaFree(c->mw_tmp);
        c->mw_tmp = nullptr;
        c->mw_tmp_n = 0;
        CK(c, cudaMalloc(&c->mw_tmp, sizeof(int64_t) * need));
        c->mw_tmp_n = need;
      }
      CK(c, launch_renumber(dst.id, c->np, kept, c->mw_tmp, c->stream));
      // the tile ranges of the next step come from this binning: keep them
    }
    c->pcur = 1 - c->pcur;
    c->steps_since_sort = 0;
    c->np = kept;
  }
  c->mw_origin = (c->mw_origin + 1) % c->g.n[0];
  ++c->mw_shifts;
  ++c->epoch;
  return PIC_OK;
}

// after every step: the shifts the window owes (one each time c t since its
// start crosses a multiple of dx1)
pic_status window_after_step(pic_ctx* c) {
  if (c->mw_start < 0) return PIC_OK;
  ++c->mw_steps;
  if (c->mw_steps <= c->mw_start) return PIC_OK;
  const int64_t target =
      (int64_t)floor((double)(c->mw_steps - c->mw_start) * c->dt / c->g.dx[0] + 1e-9);
  while (c->mw_shifts < target) {
    pic_status st = window_shift(c);
    if (st != PIC_OK) return st;
  }
  return PIC_OK;
}

// The graph replaying two steps from the current (field parity, particle
// buffer), captured on first use; nullptr if capture is not possible.
cudaGraphExec_t step_pair_graph(pic_ctx* c) {
  if (c->graphs_off) return nullptr;
  for (auto& g : c->sgraph)
    if (g.exec && g.epoch == c->epoch && g.cur == c->cur && g.pcur == c->pcur) return g.exec;
  // capture: run the two steps' launches into a graph, then restore the host
  // bookkeeping they advanced (it is advanced again at each replay)
  const int cur = c->cur, pcur = c->pcur, sss = c->steps_since_sort;
  const int64_t done = c->steps_done;
  cudaGraph_t gr = nullptr;
  cudaGraphExec_t ex = nullptr;
  bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    pic_status s1 = step_once(c);
    pic_status s2 = s1 == PIC_OK ? step_once(c) : s1;
    ok = cudaStreamEndCapture(c->stream, &gr) == cudaSuccess && s1 == PIC_OK && s2 == PIC_OK &&
         gr && cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
  }
  if (gr) cudaGraphDestroy(gr);
  cudaGetLastError();  // a failed capture leaves no sticky error
  c->cur = cur;
  c->pcur = pcur;
  c->steps_since_sort = sss;
  c->steps_done = done;
  if (!ok) {
    if (ex) cudaGraphExecDestroy(ex);
    c->graphs_off = true;
    return nullptr;
  }
  // keep it in a free slot, or in place of one from an older epoch
  int slot = 0;
  for (int k = 0; k < 4; ++k)
    if (!c->sgraph[k].exec || c->sgraph[k].epoch != c->epoch) {
      slot = k;
      break;
    }
  if (c->sgraph[slot].exec) cudaGraphExecDestroy(c->sgraph[slot].exec);
  c->sgraph[slot] = pic_ctx::StepGraph{ex, cur, pcur, c->epoch};
  return ex;
}

pic_status pic_step(pic_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return fail(c, PIC_ERR_ARG, "bad arguments");
  CK(c, cudaSetDevice(c->device));
  int64_t s = 0;
  while (s < nsteps) {
    // pairs of steps without a re-binning between them replay a captured graph
    // (launch overhead dominates small grids); timing runs take plain launches
    const int64_t room = std::min<int64_t>(nsteps - s, c->sort_interval - c->steps_since_sort);
    if (c->mw_start >= 0 || c->spec) {   // moving window or spectral path: one step at a time
      pic_status st = step_once(c);
      if (st == PIC_OK) st = window_after_step(c);
      if (st != PIC_OK) return st;
      ++s;
      continue;
    }
    if (!c->timing && room >= 2) {
      cudaGraphExec_t ex = step_pair_graph(c);
      if (ex) {
        const int64_t pairs = room / 2;
        for (int64_t k = 0; k < pairs; ++k) CK(c, cudaGraphLaunch(ex, c->stream));
        c->steps_since_sort += (int)(2 * pairs);
        c->steps_done += 2 * pairs;
        s += 2 * pairs;
        continue;
      }
    }
    pic_status st = step_once(c);
    if (st != PIC_OK) return st;
    ++s;
  }
  return PIC_OK;
}

pic_status pic_read_particles(pic_ctx* c, double* x, double* u, double* w, int on_device) {
  if (!c) return PIC_ERR_ARG;
  CK(c, cudaSetDevice(c->device));
  const int64_t n = c->np;
  const int nd = c->grid.ndim;
  if (n == 0) return PIC_OK;
  if (on_device) {
    CK(c, launch_unpermute(c->parts[c->pcur], nd, n, x, u, w, c->g.len, c->stream));
    return PIC_OK;
  }
  if (c->rbuf_n < n * (nd + 4)) {
    cudaFree(c->rbuf);
    c->rbuf = nullptr;
    c->rbuf_n = 0;
    if (cudaMalloc(&c->rbuf, sizeof(double) * n * (nd + 4)) != cudaSuccess)
      return fail(c, PIC_ERR_OOM, "particle read-back buffer");
    c->rbuf_n = n * (nd + 4);
  }
  double* tmp = c->rbuf;
  double *dx = tmp, *du = tmp + nd * n, *dw = tmp + (nd + 3) * n;
  cudaError_t e = launch_unpermute(c->parts[c->pcur], nd, n, dx, du, dw, c->g.len, c->stream);
  if (e == cudaSuccess && x) e = cudaMemcpyAsync(x, dx, sizeof(double) * nd * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && w) e = cudaMemcpyAsync(w, dw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  CK(c, e);
  return check_err_word(c);
}

pic_status pic_set_energy_gain(pic_ctx* c, int on) {
  if (!c) return PIC_ERR_ARG;
  CK(c, cudaSetDevice(c->device));
  CK(c, cudaStreamSynchronize(c->stream));
  ++c->epoch;  // the particle pointers change: captured step graphs are stale
  for (int s = 0; s < 2; ++s) {
    PartPtrs& p = c->parts[s];
    cudaFree(p.wl);
    cudaFree(p.wd);
    p.wl = p.wd = nullptr;
  }
  c->gain = on != 0;
  if (!c->gain || c->cap == 0) return PIC_OK;
  for (int s = 0; s < 2; ++s) {
    PartPtrs& p = c->parts[s];
    CK(c, cudaMalloc(&p.wl, sizeof(double) * c->cap));
    CK(c, cudaMalloc(&p.wd, sizeof(double) * c->cap));
    CK(c, cudaMemsetAsync(p.wl, 0, sizeof(double) * c->cap, c->stream));
    CK(c, cudaMemsetAsync(p.wd, 0, sizeof(double) * c->cap, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_read_energy_gain(pic_ctx* c, double* w_lwfa, double* w_dla) {
  if (!c || !w_lwfa || !w_dla) return fail(c, PIC_ERR_ARG, "null argument");
  if (!c->gain) return fail(c, PIC_ERR_STATE, "energy-gain integrals are off (pic_set_energy_gain)");
  CK(c, cudaSetDevice(c->device));
  const int64_t n = c->np;
  if (n == 0) return PIC_OK;
  if (c->rbuf_n < 2 * n) {
    cudaFree(c->rbuf);
    c->rbuf = nullptr;
    c->rbuf_n = 0;
    if (cudaMalloc(&c->rbuf, sizeof(double) * 2 * n) != cudaSuccess)
      return fail(c, PIC_ERR_OOM, "read-back buffer");
    c->rbuf_n = 2 * n;
  }
  cudaError_t e = launch_unpermute_gain(c->parts[c->pcur], n, c->rbuf, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w_lwfa, c->rbuf, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w_dla, c->rbuf + n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  CK(c, e);
  return check_err_word(c);
}

pic_status pic_set_spectral(pic_ctx* c, int nbins, const double* kE1, const double* kB1,
                            double slope0) {
  if (!c) return PIC_ERR_ARG;
  CK(c, cudaSetDevice(c->device));
  CK(c, cudaStreamSynchronize(c->stream));
  ++c->epoch;
  if (nbins == 0) {
    spectral_free(c->spec);
    c->spec = nullptr;
    return PIC_OK;
  }
  if (c->grid.precision != PIC_FP64)
    return fail(c, PIC_ERR_STATE, "the spectral field path runs in FP64 contexts");
  for (int k = 0; k < 3; ++k)
    if (!c->bbar[k] && cudaMalloc(&c->bbar[k], sizeof(double) * c->g.ncell) != cudaSuccess)
      return fail(c, PIC_ERR_OOM, "time-centred B arrays");
  pic_status st = spectral_setup(c, nbins, kE1, kB1, slope0);
  if (st != PIC_OK)
    return fail(c, st, st == PIC_ERR_ARG ? "nbins must be n1/2 + 1, finite symbols, [k]_B1 != 0 "
                                           "for k > 0, slope0 > 0"
                                         : "cuFFT plan or buffer set-up failed");
  return PIC_OK;
}

pic_status pic_set_moving_window(pic_ctx* c, int64_t start_step) {
  if (!c) return PIC_ERR_ARG;
  if (start_step >= 0 && c->grid.ndim != 2 && c->grid.ndim != 3) return PIC_ERR_ARG;
  c->mw_start = start_step < 0 ? -1 : start_step;
  c->mw_steps = 0;
  c->mw_shifts = 0;
  return PIC_OK;
}

pic_status pic_get_window(pic_ctx* c, int64_t* origin, int64_t* shifts) {
  if (!c || !origin || !shifts) return fail(c, PIC_ERR_ARG, "null argument");
  *origin = c->mw_origin;
  *shifts = c->mw_shifts;
  return PIC_OK;
}

pic_status pic_sync(pic_ctx* c) {
  if (!c) return PIC_ERR_ARG;
  CK(c, cudaSetDevice(c->device));
  CK(c, cudaStreamSynchronize(c->stream));
  return check_err_word(c);
}

pic_status pic_get_info(pic_ctx* c, pic_info* info) {
  if (!c || !info) return fail(c, PIC_ERR_ARG, "null argument");
  CK(c, cudaSetDevice(c->device));
  memset(info, 0, sizeof *info);
  info->sort_interval = c->sort_interval;
  for (int d = 0; d < 3; ++d) {
    info->tile[d] = c->ptile.t[d];
    info->guard[d] = c->ptile.g[d];
  }
  info->n_particles = c->np;
  info->steps_done = c->steps_done;
  unsigned long long sc = 0;
  if (c->np > 0) {
    CK(c, cudaMemcpyAsync(&sc, c->bins.strag_count, sizeof sc, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  info->last_stragglers = (int64_t)sc;
  info->correction_active = c->corr ? 1 : 0;
  info->cfl_lhs = c->cfl_lhs;
  info->cfl_sufficient_dt = c->cfl_suff;
  info->kernels_per_step = 1 + (c->np > 0 ? (c->grid.ndim == 3 ? 3 : 2) : 0) + (c->corr ? 1 : 0);
  return PIC_OK;
}

pic_status pic_set_timing(pic_ctx* c, int enable) {
  if (!c) return PIC_ERR_ARG;
  CK(c, cudaSetDevice(c->device));
  CK(c, cudaStreamSynchronize(c->stream));
  for (auto& t : c->tev) {
    c->evpool.push_back(t.second.first);
    c->evpool.push_back(t.second.second);
  }
  c->tev.clear();
  c->t_launches = 0;
  c->t_steps = 0;
  c->timing = enable != 0;
  return PIC_OK;
}

pic_status pic_get_timing(pic_ctx* c, pic_timing* out) {
  if (!c || !out) return fail(c, PIC_ERR_ARG, "null argument");
  CK(c, cudaSetDevice(c->device));
  CK(c, cudaStreamSynchronize(c->stream));
  double ms[5] = {0, 0, 0, 0, 0};
  for (auto& t : c->tev) {
    float v = 0;
    CK(c, cudaEventElapsedTime(&v, t.second.first, t.second.second));
    ms[t.first] += v;
  }
  out->ms_rebin = ms[0];
  out->ms_particles = ms[1];
  out->ms_stragglers = ms[2];
  out->ms_correction = ms[3];
  out->ms_fields = ms[4];
  out->launches = c->t_launches;
  out->steps = c->t_steps;
  return PIC_OK;
}

pic_status pic_set_sort_interval(pic_ctx* c, int interval) {
  if (!c || interval < 1) return fail(c, PIC_ERR_ARG, "interval must be >= 1");
  c->sort_interval = interval;
  return PIC_OK;
}

pic_status pic_set_field_tile(pic_ctx* c, int t1, int t2, int t3, int threads, int staging) {
  if (!c) return PIC_ERR_ARG;
  if (threads != 128 && threads != 256 && threads != 512)
    return fail(c, PIC_ERR_ARG, "threads must be 128, 256 or 512");
  if (t1 < 1 || t2 < 1 || t3 < 1 || t1 > 4096 || t2 > 256 || t3 > 256 ||
      (c->grid.ndim == 2 && t3 != 1))
    return fail(c, PIC_ERR_ARG, "field tile extents out of range (2D grids need t3 = 1)");
  if (staging < 0 || staging > 2) return fail(c, PIC_ERR_ARG, "staging must be 0, 1 or 2");
  if (t1 % (16 / (int)c->tsize) != 0)
    return fail(c, PIC_ERR_ARG, "t1 must be a multiple of 16 bytes of the field type");
  if (field_tile_smem_elems(c->grid.ndim, t1, t2, t3, c->M, (int)c->tsize) * c->tsize > 200 * 1024)
    return fail(c, PIC_ERR_ARG, "field tile does not fit in shared memory");
  c->ftile.t[0] = t1;
  c->ftile.t[1] = t2;
  c->ftile.t[2] = t3;
  c->ftile.threads = threads;
  c->ftile.staging = staging;
  ++c->epoch;
  return PIC_OK;
}

pic_status pic_set_field_strip(pic_ctx* c, int width, int rows, int warps, int stages) {
  if (!c) return PIC_ERR_ARG;
  if (width < 1 || width % (16 / (int)c->tsize) != 0 || width > 4096)
    return fail(c, PIC_ERR_ARG, "strip width must be a positive multiple of 16 bytes of the field type");
  if (rows < 0 || warps < 1 || warps > 16 || stages < 2 || stages > 8)
    return fail(c, PIC_ERR_ARG, "rows >= 0, 1 <= warps <= 16, 2 <= stages <= 8");
  const int V = 16 / (int)c->tsize;
  const int MT = stencil_mt(c->M);
  const Reach R(MT, V);
  if (c->grid.ndim == 3 && warps > 8)
    return fail(c, PIC_ERR_ARG, "3D strips take at most 8 warps (planes) per CTA");
  size_t elems;
  if (c->grid.ndim == 3 && warps > 1)
    elems = (size_t)planes3_cta_elems(warps, width, R.WE(width, V), R.WB(width, V), stages);
  else if (c->grid.ndim == 3)
    elems = (size_t)stages * (9 * R.WE(width, V) + 6 * R.WB(width, V) + 3 * width) + 8 * R.WB(width, V);
  else
    elems = warps * ((size_t)stages * 3 * (R.WE(width, V) + R.WB(width, V)) + 6 * R.WB(width, V));
  if (elems * c->tsize + 128 > 200 * 1024)
    return fail(c, PIC_ERR_ARG, "strip rows do not fit in shared memory");
  c->ftile.sw = width;
  c->ftile.rows = rows;
  c->ftile.warps = warps;
  c->ftile.stages = stages;
  ++c->epoch;
  return PIC_OK;
}

pic_status pic_set_correction_path(pic_ctx* c, int path) {
  if (!c) return PIC_ERR_ARG;
  if (path < 0 || path > 3) return fail(c, PIC_ERR_ARG, "correction path must be 0..3");
  if (path == 1 && c->corr &&
      (size_t)(2 * ceil_to(c->taps_n, 16 / (int)c->tsize) + ceil_to(c->g.n[0], 16 / (int)c->tsize)) *
              c->tsize > 200 * 1024)
    return fail(c, PIC_ERR_ARG, "an x1 row and the correction taps do not fit in shared memory");
  if (path == 2 && c->corr && (size_t)(1024 + 2 * c->taps_n) * c->tsize > 200 * 1024)
    return fail(c, PIC_ERR_ARG, "the correction taps do not fit in shared memory");
  c->corr_path = path;
  ++c->epoch;
  return PIC_OK;
}

pic_status pic_laser_profile(int n1, double dx1, double dt, const pic_coeffs* co,
                             const pic_laser* L, double* e2, double* b3) {
  if (!co || !L || !e2 || !b3 || !co->cE || !co->cB || n1 < 1 || !(dx1 > 0) || !(dt > 0) ||
      co->M < 1 || co->M > PIC_MAX_M)
    return PIC_ERR_ARG;
  if (!(L->L_env > 0) || L->L_env > n1 * dx1 || !isfinite(L->a0) || !(L->k0 > 0))
    return PIC_ERR_ARG;
  laser_profiles(n1, dx1, dt, co->M, co->cE, co->cB, *L, e2, b3);
  return PIC_OK;
}

pic_status pic_correction_taps(int n1, double dx1, int M, const double* cB, double* taps,
                               int* lo, int* count) {
  if (!cB || !taps || !lo || !count || n1 < 1 || M < 1 || M > PIC_MAX_M || !(dx1 > 0))
    return PIC_ERR_ARG;
  std::vector<double> t;
  int l = 0;
  if (!inv_circulant_taps(n1, dx1, M, cB, t, l)) return PIC_ERR_ARG;
  for (size_t q = 0; q < t.size(); ++q) taps[q] = t[q];
  *lo = l;
  *count = (int)t.size();
  return PIC_OK;
}

pic_status pic_state_size(pic_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(c, PIC_ERR_ARG, "null argument");
  *bytes = state_bytes(c);
  return PIC_OK;
}

pic_status pic_save_state(pic_ctx* c, void* buf, size_t bytes) {
  if (!c || !buf) return fail(c, PIC_ERR_ARG, "null argument");
  if (bytes < state_bytes(c)) return fail(c, PIC_ERR_ARG, "state buffer too small (pic_state_size)");
  pic_status st = pic_sync(c);  // a latched device error is reported, not saved
  if (st != PIC_OK) return st;
  unsigned char* p = static_cast<unsigned char*>(buf);
  StateHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kStateMagic, 8);
  h.version = 1;
  h.ndim = c->grid.ndim;
  h.precision = c->grid.precision;
  h.M = c->M;
  for (int d = 0; d < 3; ++d) {
    h.n[d] = c->g.n[d];
    h.dx[d] = c->g.dx[d];
  }
  h.dt = c->dt;
  h.qm = c->qm;
  for (int j = 0; j < PIC_MAX_M; ++j) {
    h.cE[j] = c->cE[j];
    h.cB[j] = c->cB[j];
  }
  h.np = c->np;
  h.steps_done = c->steps_done;
  h.field_bytes = 6 * (uint64_t)c->g.ncell * c->tsize;
  h.part_bytes = (uint64_t)c->np * (uint64_t)(c->grid.ndim + 4) * sizeof(double);
  memset(p, 0, kStateHdr);
  memcpy(p, &h, sizeof h);
  const size_t fb = (size_t)c->g.ncell * c->tsize;
  unsigned char* q = p + kStateHdr;
  for (int k = 0; k < 3; ++k)
    CK(c, cudaMemcpyAsync(q + k * fb, c->fe[c->cur][k], fb, cudaMemcpyDeviceToHost, c->stream));
  for (int k = 0; k < 3; ++k)
    CK(c, cudaMemcpyAsync(q + (3 + k) * fb, c->fb[c->cur][k], fb, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (c->np > 0) {
    double* x = reinterpret_cast<double*>(q + 6 * fb);
    double* u = x + (size_t)c->grid.ndim * c->np;
    double* w = u + 3 * (size_t)c->np;
    st = pic_read_particles(c, x, u, w, 0);
    if (st != PIC_OK) return st;
  }
  return PIC_OK;
}

pic_status pic_load_state(pic_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return fail(c, PIC_ERR_ARG, "null argument");
  if (bytes < kStateHdr) return fail(c, PIC_ERR_ARG, "state buffer too small");
  const unsigned char* p = static_cast<const unsigned char*>(buf);
  StateHeader h;
  memcpy(&h, p, sizeof h);
  if (memcmp(h.magic, kStateMagic, 8) != 0 || h.version != 1)
    return fail(c, PIC_ERR_ARG, "not a saved state");
  bool same = h.ndim == c->grid.ndim && h.precision == c->grid.precision && h.M == c->M &&
              h.dt == c->dt;
  for (int d = 0; d < 3; ++d) same = same && h.n[d] == c->g.n[d] && h.dx[d] == c->g.dx[d];
  for (int j = 0; j < PIC_MAX_M; ++j) same = same && h.cE[j] == c->cE[j] && h.cB[j] == c->cB[j];
  if (!same) return fail(c, PIC_ERR_ARG, "state was saved from a different grid, time step or solver");
  const size_t fb = (size_t)c->g.ncell * c->tsize;
  if (h.np < 0 || h.field_bytes != 6 * (uint64_t)fb ||
      h.part_bytes != (uint64_t)h.np * (uint64_t)(c->grid.ndim + 4) * sizeof(double) ||
      bytes < kStateHdr + h.field_bytes + h.part_bytes)
    return fail(c, PIC_ERR_ARG, "state buffer truncated or inconsistent");
  CK(c, cudaSetDevice(c->device));
  CK(c, cudaStreamSynchronize(c->stream));
  const unsigned char* q = p + kStateHdr;
  for (int k = 0; k < 3; ++k)
    CK(c, cudaMemcpyAsync(c->fe[c->cur][k], q + k * fb, fb, cudaMemcpyHostToDevice, c->stream));
  for (int k = 0; k < 3; ++k)
    CK(c, cudaMemcpyAsync(c->fb[c->cur][k], q + (3 + k) * fb, fb, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const double* x = reinterpret_cast<const double*>(q + 6 * fb);
  const double* u = x + (size_t)c->grid.ndim * h.np;
  const double* w = u + 3 * (size_t)h.np;
  pic_status st = pic_load_particles(c, h.np, h.np ? x : nullptr, h.np ? u : nullptr,
                                     h.np ? w : nullptr, h.qm, 0);
  if (st != PIC_OK) return st;
  c->steps_done = h.steps_done;
  ++c->epoch;
  return PIC_OK;
}

}  // extern "C"
