// spectral.cu -- the spectral x1 field path of libpic (FP64).
//
// The paper builds its solver from k-space operators: [k]_E1 in Faraday's law
// and [k]_B1 in Ampere's law (Sec. 3.1, Eqs. (11)-(15)), which an FFT-based
// solver can apply directly (Sec. 1, Sec. 3.1, Sec. 4.1) before the App. B
// stencils approximate them.  Here the leapfrog step of Eq. (1) takes its x1
// derivatives in Fourier space along x1 only, row by row:
//   d1 f (integer -> half-integer node) = IFFT( i [k]_E1 e^{+i k dx1/2} FFT(f) ),
//   d1 f (half-integer -> integer node) = IFFT( i [k]_B1 e^{-i k dx1/2} FFT(f) ),
// while the x2 and x3 derivatives stay Yee differences in real space; the x1
// current correction of Sec. 3.3 is the multiplication of the J1 row spectrum by
// [k]_Yee/[k]_B1, as the paper states it.  The transforms are batched real-to-
// complex / complex-to-real cuFFT transforms over all rows (a library FFT, like a
// library GEMM); the symbol multiplications and the real-space updates are this
// file's kernels.  The caller gives [k]_E1, [k]_B1 at the n1/2 + 1 non-negative
// x1 wavenumbers k_m = 2 pi m / (n1 dx1).
#include <cufft.h>
#include <math.h>

#include <vector>

#include "common.cuh"
#include "ctx.cuh"

using namespace pic;

struct SpectralState {
  int n1 = 0, nh = 0;
  int64_t rows = 0;
  cufftHandle fwd = 0, inv = 0;
  bool plans = false;
  cufftDoubleComplex* c[2] = {nullptr, nullptr};  // rows x nh each
  double* d[2] = {nullptr, nullptr};              // ncell each: x1 derivatives
  cufftDoubleComplex* symE = nullptr;             // i [k]_E1 e^{+i k dx1/2} / n1
  cufftDoubleComplex* symB = nullptr;             // i [k]_B1 e^{-i k dx1/2} / n1
  double* ratio = nullptr;                        // [k]_Yee/[k]_B1 / n1, null: identity
};

namespace {

__global__ void sym_mul2_kernel(cufftDoubleComplex* a, cufftDoubleComplex* b,
                                const cufftDoubleComplex* sym, int nh, int64_t total) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const cufftDoubleComplex s = sym[q % nh];
    const cufftDoubleComplex x = a[q], y = b[q];
    a[q] = make_cuDoubleComplex(x.x * s.x - x.y * s.y, x.x * s.y + x.y * s.x);
    b[q] = make_cuDoubleComplex(y.x * s.x - y.y * s.y, y.x * s.y + y.y * s.x);
  }
}

__global__ void ratio_mul_kernel(cufftDoubleComplex* a, const double* r, int nh, int64_t total) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double s = r[q % nh];
    a[q].x *= s;
    a[q].y *= s;
  }
}

__device__ __forceinline__ int64_t cell(int i, int j, int k, int n1, int n2) {
  return ((int64_t)k * n2 + j) * n1 + i;
}

// Faraday, Eq. (1): B^{n+1/2} = B^{n-1/2} - dt curl_E E^n with the spectral x1
// derivatives d1e2 = d1 E2, d1e3 = d1 E3 (at the B nodes) and Yee x2/x3
// differences; also the time-centred B^n = (B^{n-1/2} + B^{n+1/2})/2 (Eq. (7)).
__global__ void faraday_spec_kernel(FieldPtrs<double> f, double* bo1, double* bo2, double* bo3,
                                    double* bb1, double* bb2, double* bb3, const double* d1e2,
                                    const double* d1e3, int n1, int n2, int n3, double dt,
                                    double y2, double y3) {
  const int64_t nc = (int64_t)n1 * n2 * n3;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nc;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const int64_t r = q / n1;
    const int j = (int)(r % n2), k = (int)(r / n2);
    const int64_t qj = cell(i, j + 1 == n2 ? 0 : j + 1, k, n1, n2);
    const int64_t qk = cell(i, j, k + 1 == n3 ? 0 : k + 1, n1, n2);
    const double d2E3 = f.e[2][qj] - f.e[2][q], d2E1 = f.e[0][qj] - f.e[0][q];
    const double d3E2 = n3 > 1 ? f.e[1][qk] - f.e[1][q] : 0.0;
    const double d3E1 = n3 > 1 ? f.e[0][qk] - f.e[0][q] : 0.0;
    const double c1 = y2 * d2E3 - y3 * d3E2;
    const double c2 = y3 * d3E1 - dt * d1e3[q];
    const double c3 = dt * d1e2[q] - y2 * d2E1;
    const double b1 = f.b[0][q], b2 = f.b[1][q], b3 = f.b[2][q];
    const double n1v = b1 - c1, n2v = b2 - c2, n3v = b3 - c3;
    bo1[q] = n1v;
    bo2[q] = n2v;
    bo3[q] = n3v;
    bb1[q] = 0.5 * (b1 + n1v);
    bb2[q] = 0.5 * (b2 + n2v);
    bb3[q] = 0.5 * (b3 + n3v);
  }
}

// Ampere, Eq. (1): E^{n+1} = E^n + dt (curl_B B^{n+1/2} - J) with d1b2 = d1 B2,
// d1b3 = d1 B3 (at the E nodes) and Yee x2/x3 differences.
__global__ void ampere_spec_kernel(const double* e1, const double* e2, const double* e3,
                                   const double* b1, const double* b2, const double* b3,
                                   const double* j1, const double* j2, const double* j3,
                                   double* eo1, double* eo2, double* eo3, const double* d1b2,
                                   const double* d1b3, int n1, int n2, int n3, double dt,
                                   double y2, double y3) {
  const int64_t nc = (int64_t)n1 * n2 * n3;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nc;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const int64_t r = q / n1;
    const int j = (int)(r % n2), k = (int)(r / n2);
    const int64_t qj = cell(i, j == 0 ? n2 - 1 : j - 1, k, n1, n2);
    const int64_t qk = cell(i, j, k == 0 ? n3 - 1 : k - 1, n1, n2);
    const double d2B3 = b3[q] - b3[qj], d2B1 = b1[q] - b1[qj];
    const double d3B2 = n3 > 1 ? b2[q] - b2[qk] : 0.0;
    const double d3B1 = n3 > 1 ? b1[q] - b1[qk] : 0.0;
    eo1[q] = e1[q] + ((y2 * d2B3 - y3 * d3B2) - dt * j1[q]);
    eo2[q] = e2[q] + ((y3 * d3B1 - dt * d1b3[q]) - dt * j2[q]);
    eo3[q] = e3[q] + ((dt * d1b2[q] - y2 * d2B1) - dt * j3[q]);
  }
}

inline unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

cudaError_t fft_err(cufftResult r) {
  return r == CUFFT_SUCCESS ? cudaSuccess
                            : (r == CUFFT_ALLOC_FAILED ? cudaErrorMemoryAllocation : cudaErrorUnknown);
}

// x1 derivatives of two arrays: d[0] = d1 a, d[1] = d1 b with the symbol sym
cudaError_t x1_derivs(SpectralState* S, const double* a, const double* b,
                      const cufftDoubleComplex* sym, cudaStream_t st) {
  cudaError_t e = fft_err(cufftExecD2Z(S->fwd, const_cast<double*>(a), S->c[0]));
  if (e == cudaSuccess) e = fft_err(cufftExecD2Z(S->fwd, const_cast<double*>(b), S->c[1]));
  if (e != cudaSuccess) return e;
  const int64_t tot = S->rows * S->nh;
  sym_mul2_kernel<<<blocks_for(tot), 256, 0, st>>>(S->c[0], S->c[1], sym, S->nh, tot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = fft_err(cufftExecZ2D(S->inv, S->c[0], S->d[0]));
  if (e == cudaSuccess) e = fft_err(cufftExecZ2D(S->inv, S->c[1], S->d[1]));
  return e;
}

}  // namespace

void spectral_free(SpectralState* S) {
  if (!S) return;
  if (S->plans) {
    cufftDestroy(S->fwd);
    cufftDestroy(S->inv);
  }
  for (int k = 0; k < 2; ++k) {
    cudaFree(S->c[k]);
    cudaFree(S->d[k]);
  }
  cudaFree(S->symE);
  cudaFree(S->symB);
  cudaFree(S->ratio);
  delete S;
}

pic_status spectral_setup(pic_ctx* c, int nbins, const double* kE1, const double* kB1,
                          double slope0) {
  const int n1 = c->g.n[0], nh = n1 / 2 + 1;
  if (nbins != nh || !kE1 || !kB1 || !(slope0 > 0)) return PIC_ERR_ARG;
  for (int m = 0; m < nh; ++m)
    if (!isfinite(kE1[m]) || !isfinite(kB1[m]) || (m > 0 && kB1[m] == 0.0)) return PIC_ERR_ARG;
  SpectralState* S = new SpectralState();
  S->n1 = n1;
  S->nh = nh;
  S->rows = c->g.ncell / n1;
  auto bad = [&](pic_status s) {
    spectral_free(S);
    return s;
  };
  int n = n1;
  if (S->rows > INT32_MAX) return bad(PIC_ERR_ARG);
  if (cufftPlanMany(&S->fwd, 1, &n, nullptr, 1, n1, nullptr, 1, nh, CUFFT_D2Z, (int)S->rows) !=
      CUFFT_SUCCESS)
    return bad(PIC_ERR_CUDA);
  if (cufftPlanMany(&S->inv, 1, &n, nullptr, 1, nh, nullptr, 1, n1, CUFFT_Z2D, (int)S->rows) !=
      CUFFT_SUCCESS) {
    cufftDestroy(S->fwd);
    return bad(PIC_ERR_CUDA);
  }
  S->plans = true;
  if (cufftSetStream(S->fwd, c->stream) != CUFFT_SUCCESS ||
      cufftSetStream(S->inv, c->stream) != CUFFT_SUCCESS)
    return bad(PIC_ERR_CUDA);
  for (int k = 0; k < 2; ++k) {
    if (cudaMalloc(&S->c[k], sizeof(cufftDoubleComplex) * S->rows * nh) != cudaSuccess ||
        cudaMalloc(&S->d[k], sizeof(double) * c->g.ncell) != cudaSuccess)
      return bad(PIC_ERR_OOM);
  }
  // symbols at k_m = 2 pi m / (n1 dx1), with the 1/n1 of the unnormalised inverse
  const double dx = c->g.dx[0];
  std::vector<cufftDoubleComplex> sE(nh), sB(nh);
  std::vector<double> rt(nh);
  bool ident = true;
  for (int m = 0; m < nh; ++m) {
    const double k = 2.0 * M_PI * m / (n1 * dx), th = 0.5 * k * dx;
    sE[m] = make_cuDoubleComplex(-sin(th) * kE1[m] / n1, cos(th) * kE1[m] / n1);
    sB[m] = make_cuDoubleComplex(sin(th) * kB1[m] / n1, cos(th) * kB1[m] / n1);
    const double r = m == 0 ? 1.0 / slope0 : (sin(th) / (0.5 * dx)) / kB1[m];
    ident = ident && fabs(r - 1.0) <= 1e-15;
    rt[m] = r / n1;
  }
  if (cudaMalloc(&S->symE, sizeof(cufftDoubleComplex) * nh) != cudaSuccess ||
      cudaMalloc(&S->symB, sizeof(cufftDoubleComplex) * nh) != cudaSuccess)
    return bad(PIC_ERR_OOM);
  if (cudaMemcpy(S->symE, sE.data(), sizeof(cufftDoubleComplex) * nh, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(S->symB, sB.data(), sizeof(cufftDoubleComplex) * nh, cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return bad(PIC_ERR_CUDA);
  if (!ident) {
    if (cudaMalloc(&S->ratio, sizeof(double) * nh) != cudaSuccess) return bad(PIC_ERR_OOM);
    if (cudaMemcpy(S->ratio, rt.data(), sizeof(double) * nh, cudaMemcpyHostToDevice) != cudaSuccess)
      return bad(PIC_ERR_CUDA);
  }
  spectral_free(c->spec);
  c->spec = S;
  return PIC_OK;
}

cudaError_t spectral_faraday(pic_ctx* c, const FieldPtrs<double>& f, double* const* bo,
                             double* const* bb) {
  SpectralState* S = c->spec;
  cudaError_t e = x1_derivs(S, f.e[1], f.e[2], S->symE, c->stream);   // d1 E2, d1 E3
  if (e != cudaSuccess) return e;
  const int n3 = c->grid.ndim == 3 ? c->g.n[2] : 1;
  faraday_spec_kernel<<<blocks_for(c->g.ncell), 256, 0, c->stream>>>(
      f, bo[0], bo[1], bo[2], bb[0], bb[1], bb[2], S->d[0], S->d[1], c->g.n[0], c->g.n[1], n3,
      c->dt, c->dt / c->g.dx[1], n3 > 1 ? c->dt / c->g.dx[2] : 0.0);
  return cudaGetLastError();
}

cudaError_t spectral_correct_j1(pic_ctx* c, double* j1) {
  SpectralState* S = c->spec;
  if (!S->ratio) return cudaSuccess;
  cudaError_t e = fft_err(cufftExecD2Z(S->fwd, j1, S->c[0]));
  if (e != cudaSuccess) return e;
  const int64_t tot = S->rows * S->nh;
  ratio_mul_kernel<<<blocks_for(tot), 256, 0, c->stream>>>(S->c[0], S->ratio, S->nh, tot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return fft_err(cufftExecZ2D(S->inv, S->c[0], j1));
}

cudaError_t spectral_ampere(pic_ctx* c, const FieldPtrs<double>& f, double* const* bnew,
                            double* const* eo) {
  SpectralState* S = c->spec;
  cudaError_t e = x1_derivs(S, bnew[1], bnew[2], S->symB, c->stream);   // d1 B2, d1 B3
  if (e != cudaSuccess) return e;
  const int n3 = c->grid.ndim == 3 ? c->g.n[2] : 1;
  ampere_spec_kernel<<<blocks_for(c->g.ncell), 256, 0, c->stream>>>(
      f.e[0], f.e[1], f.e[2], bnew[0], bnew[1], bnew[2], f.j[0], f.j[1], f.j[2], eo[0], eo[1],
      eo[2], S->d[0], S->d[1], c->g.n[0], c->g.n[1], n3, c->dt, c->dt / c->g.dx[1],
      n3 > 1 ? c->dt / c->g.dx[2] : 0.0);
  return cudaGetLastError();
}
