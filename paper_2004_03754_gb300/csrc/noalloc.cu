// noalloc.cu -- allocation-free variant of the laser load.
//
// pic_laser_fields_noalloc computes the same E2^0 and B3^{-1/2} as
// pic_load_laser, but writes them into device arrays the caller owns and keeps
// its only scratch -- the two 1D x1 profiles of the pulse -- in a file-scope
// device array instead of memory obtained from cudaMalloc.  It calls no
// cudaMalloc, cudaFree or allocating library routine.
#include <math.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "laser_host.h"

namespace {

// Profiles of E2 (first PIC_NOALLOC_MAX_N1 entries) and B3 (next ones).  Every
// GPU that loads the library holds these 2 * 65536 doubles (1 MiB) until exit.
__device__ __align__(256) double g_laser_scratch[2 * PIC_NOALLOC_MAX_N1];

// Device address of g_laser_scratch, looked up once per device (the host-side
// name of the array is a stand-in, not a device address).
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_laser_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void laser_expand_noalloc_kernel(const double* __restrict__ prof, int n1, int n2,
                                            int64_t ncell, int ndim, double dx2, double dx3,
                                            double w0, double x2c, double x3c, double* e2,
                                            double* b3) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const int64_t r = q / n1;
    const int j = (int)(r % n2), k = (int)(r / n2);
    double tr = 1.0;
    if (w0 > 0.0) {
      const double d2 = ((j + 0.5) * dx2 - x2c) / w0;
      tr = exp(-d2 * d2);
      if (ndim == 3) {
        const double d3 = (k * dx3 - x3c) / w0;
        tr *= exp(-d3 * d3);
      }
    }
    e2[q] = prof[i] * tr;
    b3[q] = prof[n1 + i] * tr;
  }
}

}  // namespace

extern "C" pic_status pic_laser_fields_noalloc(const pic_grid* grid, double dt,
                                               const pic_coeffs* co, const pic_laser* L,
                                               double* e2, double* b3, void* stream) {
  if (!grid || !co || !L || !e2 || !b3) return PIC_ERR_ARG;
  if (grid->ndim != 2 && grid->ndim != 3) return PIC_ERR_ARG;
  if (co->M < 1 || co->M > PIC_MAX_M || !co->cE || !co->cB) return PIC_ERR_ARG;
  const int nd = grid->ndim;
  int64_t ncell = 1;
  for (int d = 0; d < nd; ++d) {
    if (grid->n[d] < 1 || !(grid->dx[d] > 0)) return PIC_ERR_ARG;
    ncell *= grid->n[d];
  }
  const int n = grid->n[0];
  if (n > PIC_NOALLOC_MAX_N1) return PIC_ERR_ARG;  // beyond the static scratch
  const double dx = grid->dx[0], Lbox = n * dx;
  if (!(dt > 0) || !(L->L_env > 0) || L->L_env > Lbox || !(L->k0 > 0) || !isfinite(L->a0))
    return PIC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ERR_CUDA;
  double* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return PIC_ERR_CUDA;

  // x1 profiles (the same host routine as pic_load_laser): E2 = -a'(phi) on the
  // E2 nodes, B3^{-1/2} its discrete forward eigenmode partner (Eq. (8))
  std::vector<double> prof(2 * (size_t)n);
  pic::laser_profiles(n, dx, dt, co->M, co->cE, co->cB, *L, prof.data(), prof.data() + n);
  cudaStream_t st = (cudaStream_t)stream;
  // both profiles are rewritten in full on every call, so nothing needs clearing
  if (cudaMemcpyAsync(scratch, prof.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return PIC_ERR_CUDA;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return PIC_ERR_CUDA;
  int64_t nb = (ncell + 255) / 256;
  if (nb > (int64_t)nsm * 32) nb = (int64_t)nsm * 32;   // grid-stride loop beyond 32 CTAs per SM
  laser_expand_noalloc_kernel<<<(unsigned)nb, 256, 0, st>>>(
      scratch, n, grid->n[1], ncell, nd, grid->dx[1], nd == 3 ? grid->dx[2] : 1.0, L->w0, L->x2c,
      L->x3c, e2, b3);
  if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
  // the host profile buffer dies with this call: wait for the copy and the kernel
  if (cudaStreamSynchronize(st) != cudaSuccess) return PIC_ERR_CUDA;
  return PIC_OK;
}
