// ctx.cuh -- the libpic context (internal): what pic_init allocates and the step
// machinery uses.  Shared by api.cu (the step) and adjoint.cu (reverse mode).
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"

using pic::BinBufs;
using pic::FieldTile;
using pic::GridArgs;
using pic::PartPtrs;
using pic::PartTile;
using pic::StencilArgs;

struct SpectralState;   // spectral.cu

struct pic_ctx {
  int device = 0;
  pic_grid grid{};
  GridArgs g{};
  double dt = 0;
  int M = 0;
  double cE[PIC_MAX_M] = {0}, cB[PIC_MAX_M] = {0};
  cudaStream_t stream = nullptr;
  size_t tsize = 8;
  // fields: two E/B sets (the field kernel writes the other one), J, scratch
  void* fe[2][3] = {{nullptr}};
  void* fb[2][3] = {{nullptr}};
  void* fj[3] = {nullptr};
  void* jtmp = nullptr;
  void* bbar[3] = {nullptr};  // time-centred B (3D particle step)
  double* scratch = nullptr;  // FP64 ncell, for load/read conversions
  double* rbuf = nullptr;     // particle read-back in the original order (grown on demand)
  int64_t rbuf_n = 0;
  int cur = 0;
  StencilArgs<double> sd{};
  StencilArgs<float> sf{};
  StencilArgs<pic::dfl> sdf{};  // compensated fields (PIC_COMPENSATED)
  bool corr = false;
  void* taps = nullptr;  // correction taps in the field precision
  int taps_lo = 0, taps_n = 0;
  int corr_path = 0;  // 0 automatic, 1 rows in place, 2 segments, 3 global
  FieldTile ftile{};
  // particles
  int64_t np = 0, cap = 0;
  double qm = -1.0;
  PartPtrs parts[2]{};
  int pcur = 0;
  PartTile ptile{};
  BinBufs bins{};
  int64_t bins_ntiles = 0;
  int sort_interval = 1;
  bool gain = false;  // energy-gain integrals per particle (Sec. 4.2) kept
  // moving window along x1 (Sec. 4.1): off while mw_start < 0; otherwise the
  // window moves at c from step mw_start of its own count on (mw_steps), and
  // column mw_origin is the trailing one; mw_tmp is scratch for re-numbering
  int64_t mw_start = -1, mw_steps = 0, mw_origin = 0, mw_shifts = 0;
  int64_t* mw_tmp = nullptr;
  int64_t mw_tmp_n = 0;
  // spectral x1 field path (spectral.cu); null: the finite-difference stencils
  SpectralState* spec = nullptr;
  int steps_since_sort = 0;
  int64_t steps_done = 0;
  double cfl_lhs = 0, cfl_suff = 0;
  std::string err;
  // optional event timing: pairs of events per kernel group
  bool timing = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> tev;
  std::vector<cudaEvent_t> evpool;
  int64_t t_launches = 0, t_steps = 0;
  // CUDA graphs of two consecutive steps without re-binning, one per (field
  // parity, particle buffer); dropped when the epoch changes (buffers or shapes)
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int cur = -1, pcur = -1;
    int64_t epoch = -1;
  };
  StepGraph sgraph[4];
  int64_t epoch = 0;
  bool graphs_off = false;  // set when a capture failed: plain launches from then on
};

// spectral.cu (FP64 contexts)
pic_status spectral_setup(pic_ctx* c, int nbins, const double* kE1, const double* kB1,
                          double slope0);
void spectral_free(SpectralState* s);
cudaError_t spectral_faraday(pic_ctx* c, const pic::FieldPtrs<double>& f, double* const* bo,
                             double* const* bb);
cudaError_t spectral_correct_j1(pic_ctx* c, double* j1);
cudaError_t spectral_ampere(pic_ctx* c, const pic::FieldPtrs<double>& f, double* const* bnew,
                            double* const* eo);
