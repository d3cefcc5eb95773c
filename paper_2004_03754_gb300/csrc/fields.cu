// fields.cu -- field kernels of libpic.
//
// field_step: one fused pass per tile of
//   B^{n+1/2} = B^{n-1/2} - dt d_E x E^n          (Eq. (1), App. B Eq. (B.1))
//   E^{n+1}   = E^n + dt (d_B x B^{n+1/2} - J)     (Eq. (1), App. B Eq. (B.2))
// with E^n and B^{n-1/2} staged in shared memory over the tile plus the halo the
// two wide x1 stencils need (2M-1 cells each side in x1, one cell in x2/x3).
// Each value of E, B, J is read from HBM once and E, B written once (15 values
// per cell, the algorithmic minimum); halo re-reads hit L2.
#include "common.cuh"

namespace pic {

namespace {

template <typename T>
struct OutPtrs {
  T* e[3];
  T* b[3];
};

// Periodic index for a region that may reach past the grid on either side (any
// number of periods: the loops run zero or one time except on tiny grids).
__device__ __forceinline__ int pwrap(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// Reads E^n, B^{n-1/2}, J from f and writes E^{n+1}, B^{n+1/2} to o: separate
// buffers, because neighbouring tiles read this tile's cells as their halo.
// Work is laid out row by row (one warp per x1 row segment) so that every
// global access is coalesced and no per-element division is needed.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) field_step_kernel(FieldPtrs<T> f, OutPtrs<T> o, GridArgs g,
                                                         StencilArgs<T> s, int TX, int TY,
                                                         int TZ) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int M = s.M;
  const int n1 = g.n[0], n2 = g.n[1], n3 = (NDIM == 3) ? g.n[2] : 1;
  const int ntx = (n1 + TX - 1) / TX, nty = (n2 + TY - 1) / TY;
  int tb = blockIdx.x;
  const int tx = tb % ntx;
  tb /= ntx;
  const int ty = tb % nty;
  const int tz = tb / nty;
  const int i0 = tx * TX, j0 = ty * TY, k0 = tz * TZ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

  // regions: E^n over [i0-2M+1, i0+TX+2M-1) x [j0-1, j0+TY+1) (x [k0-1, k0+TZ+1)),
  //          B over [i0-M, i0+TX+M-1) x [j0-1, j0+TY) (x [k0-1, k0+TZ))
  const int WE1 = TX + 4 * M - 2, WE2 = TY + 2, WE3 = (NDIM == 3) ? TZ + 2 : 1;
  const int WB1 = TX + 2 * M - 1, WB2 = TY + 1, WB3 = (NDIM == 3) ? TZ + 1 : 1;
  const int oE1 = i0 - 2 * M + 1, oB1 = i0 - M;
  const int nE = WE1 * WE2 * WE3, nB = WB1 * WB2 * WB3;
  T* sE = sm;            // [3][WE3][WE2][WE1]
  T* sB = sm + 3 * nE;   // [3][WB3][WB2][WB1]

  for (int row = warp; row < 3 * WE2 * WE3; row += nwarp) {
    const int l2 = row % WE2, r = row / WE2;
    const int l3 = r % WE3, c = r / WE3;
    const int gj = pwrap(j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(k0 - 1 + l3, n3) : 0;
    const T* src = f.e[c] + ((int64_t)gk * n2 + gj) * n1;
    T* dst = sE + row * WE1;
    for (int l1 = lane; l1 < WE1; l1 += 32) dst[l1] = src[pwrap(oE1 + l1, n1)];
  }
  for (int row = warp; row < 3 * WB2 * WB3; row += nwarp) {
    const int l2 = row % WB2, r = row / WB2;
    const int l3 = r % WB3, c = r / WB3;
    const int gj = pwrap(j0 - 1 + l2, n2);
    const int gk = (NDIM == 3) ? pwrap(k0 - 1 + l3, n3) : 0;
    const T* src = f.b[c] + ((int64_t)gk * n2 + gj) * n1;
    T* dst = sB + row * WB1;
    for (int l1 = lane; l1 < WB1; l1 += 32) dst[l1] = src[pwrap(oB1 + l1, n1)];
  }
  __syncthreads();

  // Faraday over the B region: B^{n+1/2} = B - dt d_E x E (coefficients pre-scaled)
  const int sE2 = WE1, sE3 = WE1 * WE2;
  const T* E1 = sE;
  const T* E2 = sE + nE;
  const T* E3 = sE + 2 * nE;
  for (int row = warp; row < WB2 * WB3; row += nwarp) {
    const int l2 = row % WB2, l3 = row / WB2;
    for (int l1 = lane; l1 < WB1; l1 += 32) {
      const int q = row * WB1 + l1;
      const int e = l3 * sE3 + l2 * sE2 + (l1 + M - 1);  // this B point in the E region
      T dE3 = 0, dE2 = 0;
      for (int m = 1; m <= M; ++m) {
        const T c = s.kE[m - 1];
        dE3 += c * (E3[e + m] - E3[e - m + 1]);
        dE2 += c * (E2[e + m] - E2[e - m + 1]);
      }
      const T d2E3 = s.y2 * (E3[e + sE2] - E3[e]);
      const T d2E1 = s.y2 * (E1[e + sE2] - E1[e]);
      T d3E2 = 0, d3E1 = 0;
      if (NDIM == 3) {
        d3E2 = s.y3 * (E2[e + sE3] - E2[e]);
        d3E1 = s.y3 * (E1[e + sE3] - E1[e]);
      }
      sB[q] -= d2E3 - d3E2;            // B1 -= dt (d2 E3 - d3 E2)
      sB[nB + q] -= d3E1 - dE3;        // B2 -= dt (d3 E1 - d^E1 E3)
      sB[2 * nB + q] -= dE2 - d2E1;    // B3 -= dt (d^E1 E2 - d2 E1)
    }
  }
  __syncthreads();

  // Ampere over the tile: E^{n+1} = E + dt (d_B x B^{n+1/2} - J); write E and B
  const int sB2 = WB1, sB3 = WB1 * WB2;
  const T* B1 = sB;
  const T* B2 = sB + nB;
  const T* B3 = sB + 2 * nB;
  const int TZe = (NDIM == 3) ? TZ : 1;
  const T dt = (T)g.dt;
  for (int row = warp; row < TY * TZe; row += nwarp) {
    const int o2 = row % TY, o3 = row / TY;
    const int gj = j0 + o2, gk = k0 + o3;
    if (gj >= n2 || (NDIM == 3 && gk >= n3)) continue;
    const int64_t rowoff = ((int64_t)gk * n2 + gj) * n1;
    for (int o1 = lane; o1 < TX; o1 += 32) {
      const int gi = i0 + o1;
      if (gi >= n1) break;
      const int b = (NDIM == 3 ? (o3 + 1) * sB3 : 0) + (o2 + 1) * sB2 + (o1 + M);
      const int e = (NDIM == 3 ? (o3 + 1) * sE3 : 0) + (o2 + 1) * sE2 + (o1 + 2 * M - 1);
      T dB3 = 0, dB2 = 0;
      for (int m = 1; m <= M; ++m) {
        const T c = s.kB[m - 1];
        dB3 += c * (B3[b + m - 1] - B3[b - m]);
        dB2 += c * (B2[b + m - 1] - B2[b - m]);
      }
      const T d2B3 = s.y2 * (B3[b] - B3[b - sB2]);
      const T d2B1 = s.y2 * (B1[b] - B1[b - sB2]);
      T d3B2 = 0, d3B1 = 0;
      if (NDIM == 3) {
        d3B2 = s.y3 * (B2[b] - B2[b - sB3]);
        d3B1 = s.y3 * (B1[b] - B1[b - sB3]);
      }
      const int64_t gidx = rowoff + gi;
      o.e[0][gidx] = E1[e] + ((d2B3 - d3B2) - dt * f.j[0][gidx]);
      o.e[1][gidx] = E2[e] + ((d3B1 - dB3) - dt * f.j[1][gidx]);
      o.e[2][gidx] = E3[e] + ((dB2 - d2B1) - dt * f.j[2][gidx]);
      o.b[0][gidx] = B1[b];
      o.b[1][gidx] = B2[b];
      o.b[2][gidx] = B3[b];
    }
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
// (symbol [k]_B1/[k]_Yee); taps[q] = g_{lo+q}, q < count.
template <typename T>
__global__ void correct_j1_kernel(const T* __restrict__ in, T* __restrict__ out, GridArgs g,
                                  const double* __restrict__ taps, int lo, int count) {
  const int n1 = g.n[0];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const T* rp = in + (q - i);
    double acc = 0.0;
    for (int m = 0; m < count; ++m) acc += taps[m] * (double)rp[wrap_index(i + lo + m, n1)];
    out[q] = (T)acc;
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

template <typename T>
cudaError_t launch_field_step(const FieldPtrs<T>& f, const FieldPtrs<T>& out, const GridArgs& g,
                              const StencilArgs<T>& s, const FieldTile& tile, cudaStream_t st) {
  OutPtrs<T> o;
  for (int c = 0; c < 3; ++c) {
    o.e[c] = out.e[c];
    o.b[c] = out.b[c];
  }
  const int TX = tile.t[0], TY = tile.t[1], TZ = (g.ndim == 3) ? tile.t[2] : 1;
  const int M = s.M;
  const size_t nE = (size_t)(TX + 4 * M - 2) * (TY + 2) * (g.ndim == 3 ? TZ + 2 : 1);
  const size_t nB = (size_t)(TX + 2 * M - 1) * (TY + 1) * (g.ndim == 3 ? TZ + 1 : 1);
  const size_t smem = 3 * (nE + nB) * sizeof(T);
  const int64_t ntiles = (int64_t)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY) *
                         (g.ndim == 3 ? (g.n[2] + TZ - 1) / TZ : 1);
  cudaError_t err;
  if (g.ndim == 3) {
    err = cudaFuncSetAttribute(field_step_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    field_step_kernel<T, 3><<<(unsigned)ntiles, 256, smem, st>>>(f, o, g, s, TX, TY, TZ);
  } else {
    err = cudaFuncSetAttribute(field_step_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (err != cudaSuccess) return err;
    field_step_kernel<T, 2><<<(unsigned)ntiles, 256, smem, st>>>(f, o, g, s, TX, TY, TZ);
  }
  return cudaGetLastError();
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

template <typename T>
cudaError_t launch_correct_j1(T* j1, T* tmp, const GridArgs& g, const double* taps, int lo,
                              int count, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(tmp, j1, sizeof(T) * g.ncell, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  correct_j1_kernel<T><<<grid_for(g.ncell), 256, 0, st>>>(tmp, j1, g, taps, lo, count);
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
                                            const FieldTile&, cudaStream_t);                \
  template cudaError_t launch_bbar<T>(const FieldPtrs<T>&, const GridArgs&,                 \
                                      const StencilArgs<T>&, double*, int, cudaStream_t);   \
  template cudaError_t launch_correct_j1<T>(T*, T*, const GridArgs&, const double*, int,    \
                                            int, cudaStream_t);                             \
  template cudaError_t launch_convert_in<T>(T*, const double*, int64_t, cudaStream_t);      \
  template cudaError_t launch_convert_out<T>(double*, const T*, int64_t, cudaStream_t);     \
  template cudaError_t launch_laser_expand<T>(const FieldPtrs<T>&, const GridArgs&,         \
                                              const double*, const double*, double, double, \
                                              double, cudaStream_t);
PIC_INST(double)
PIC_INST(float)
#undef PIC_INST

}  // namespace pic
