// adjoint.cu -- reverse mode of the PIC step (FP64) for vacuum runs.
//
// Field step (Eq. (1)): B' = B - K_E[C^E] E,  E' = E + K_B[C^B] B' (dt folded
// into the coefficients, no current).  With the Yee staggering, the transpose of
// the Faraday curl built on the d^E stencil (App. B Eq. (B.1)) is the Ampere
// curl built on the d^B form with the same coefficients, and vice versa.  So
// for the adjoint state (l_E, m_B = -l_B) one reverse step is
//   m_B'' = m_B - K_E[C^B] l_E,   l_E <- l_E + K_B[C^E] m_B'',
// i.e. the forward fused kernel with C^E and C^B exchanged.
//
// Particles: gather of E^n and of the time-centred B^n = B^{n-1/2} - (dt/2)
// K_E E^n (Eq. (7), App. A), Boris or analytic push, FP64 move and, for
// particles of non-zero weight, the Esirkepov deposit of J^{n+1/2} (Sec. 3.3).
// The reverse pass scatters the field adjoint with the gather's shape weights,
// adds the shape-derivative term to the position adjoint, differentiates the
// Boris rotation by hand (reverse order of its operations) or the analytic push
// through its smooth form, and carries the current's adjoint
//   lambda_J = -dt P^T lambda_E^{n+1}   (E^{n+1} = E^n + dt (d_B x B - P J))
// back through the deposit (deposit_vjp.cuh) into the particle's x^n and
// u^{n+1/2}.
//
// The forward trajectory is stored at checkpoints every `checkpoint_every`
// steps; each segment is recomputed (its states kept in device memory) and
// then swept backwards.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "analytic_vjp.cuh"
#include "common.cuh"
#include "ctx.cuh"
#include "deposit_vjp.cuh"
#include "particle_core.cuh"

using namespace pic;

namespace {

struct Vec3 {
  double x, y, z;
};
__device__ __forceinline__ Vec3 v3(double a, double b, double c) { return Vec3{a, b, c}; }
__device__ __forceinline__ Vec3 operator+(Vec3 a, Vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ Vec3 operator-(Vec3 a, Vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ Vec3 operator*(double s, Vec3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ Vec3 cross(Vec3 a, Vec3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// quadratic B-spline weights and their derivatives d w / d(position in cells)
__device__ __forceinline__ void bspline3_d(double d, double w[3], double dw[3]) {
  const double a = 0.5 - d, b = 0.5 + d;
  w[0] = 0.5 * a * a;
  w[1] = 0.75 - d * d;
  w[2] = 0.5 * b * b;
  dw[0] = -a;
  dw[1] = -2.0 * d;
  dw[2] = b;
}

struct AxisD {
  int bn, bh;
  double wn[3], wh[3], dwn[3], dwh[3];
};

__device__ __forceinline__ void axis_d(int li, double f, AxisD& a) {
  if (f < 0.5) {
    a.bn = li - 1;
    bspline3_d(f, a.wn, a.dwn);
  } else {
    a.bn = li;
    bspline3_d(f - 1.0, a.wn, a.dwn);
  }
  a.bh = li - 1;
  bspline3_d(f - 0.5, a.wh, a.dwh);
}

struct AdjPart {
  const double* F[6];      // forward E1 E2 E3 B1 B2 B3 (B^{n-1/2}) at step n
  const double* x;         // 2 x n  (x^n)
  const double* u;         // 3 x n  (u^{n-1/2})
  double* lu;              // 3 x n  adjoint of u
  double* lx;              // 2 x n  adjoint of x
  double* lE[3];           // adjoint of E^n (scatter target)
  double* SB[3];           // scatter of the time-centred B adjoint
  int64_t n;
  double qm;
  int pusher;              // PIC_BORIS or PIC_ANALYTIC
  const double* w;         // n weights, or null (test particles only)
  const double* lJ[3];     // lambda_E^{n+1} with P^T applied to component 1
  double jscale;           // -dt: lambda_J = jscale * lJ
};

// Deposit part of the reverse step of particle q: J^{n+1/2} depends on x^n and,
// through the move dt u/gamma and the factor w u3/gamma, on u^{n+1/2} (un, gn =
// its gamma).  Adds d<lambda_J, J>/dx^n into ldx and returns d<lambda_J, J>/du.
__device__ Vec3 deposit_adjoint(const AdjPart& A, int64_t q, const GridArgs& g, Vec3 un,
                                double gn, double ldx[2]) {
  const double w = A.w ? A.w[q] : 0.0;
  if (w == 0.0) return v3(0.0, 0.0, 0.0);
  const double uu[2] = {un.x, un.y};
  double r0[2], del[2], cf[2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    r0[d] = A.x[d * A.n + q] * g.inv_dx[d];
    del[d] = (g.dt / gn) * uu[d] * g.inv_dx[d];
    cf[d] = -w * g.dx_dt[d];
  }
  double gr[2], gd[2], gj;
  deposit_vjp<2>(A.lJ, g.n[0], g.n[1], 1, r0, del, cf, w * (un.z / gn), gr, gd, &gj);
#pragma unroll
  for (int d = 0; d < 2; ++d) ldx[d] += A.jscale * gr[d] * g.inv_dx[d];
  // d(u_k / gamma)/du = (e_k - (u_k / gamma^2) u) / gamma
  const double ig = 1.0 / gn, ig2 = ig * ig;
  const Vec3 d0 = ig * (v3(1.0, 0.0, 0.0) - (un.x * ig2) * un);
  const Vec3 d1 = ig * (v3(0.0, 1.0, 0.0) - (un.y * ig2) * un);
  const Vec3 d2 = ig * (v3(0.0, 0.0, 1.0) - (un.z * ig2) * un);
  return (A.jscale * gd[0] * g.dt * g.inv_dx[0]) * d0 + (A.jscale * gd[1] * g.dt * g.inv_dx[1]) * d1 +
         (A.jscale * gj * w) * d2;
}

// One reverse step of the test particles of a 2D run (PUSH: the pusher).
template <int PUSH>
__global__ void adjoint_particle_kernel(AdjPart A, GridArgs g, StencilArgs<double> s) {
  const int n1 = g.n[0], n2 = g.n[1];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < A.n;
       q += (int64_t)gridDim.x * blockDim.x) {
    AxisD ax[2];
    for (int d = 0; d < 2; ++d) {
      const double c = A.x[d * A.n + q] * g.inv_dx[d];
      const double fl = floor(c);
      axis_d((int)fl, c - fl, ax[d]);
    }
    GlobView<double> ve[3];
    BbarView<double, 2> vb[3];
    for (int c = 0; c < 3; ++c) {
      ve[c] = GlobView<double>{A.F[c], n1, n2, 1, n1};
      vb[c] = BbarView<double, 2>{{A.F[0], A.F[1], A.F[2]}, A.F[3 + c], c, n1, n2, 1, &s, n1};
    }
    // gather of the six components and their x-gradients (App. A)
    constexpr int half[6][2] = {{1, 0}, {0, 1}, {0, 0}, {0, 1}, {1, 0}, {1, 1}};
    double eb[6], g1[6], g2[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int b1 = half[c][0] ? ax[0].bh : ax[0].bn;
      const int b2 = half[c][1] ? ax[1].bh : ax[1].bn;
      const double* w1 = half[c][0] ? ax[0].wh : ax[0].wn;
      const double* w2 = half[c][1] ? ax[1].wh : ax[1].wn;
      const double* d1 = half[c][0] ? ax[0].dwh : ax[0].dwn;
      const double* d2 = half[c][1] ? ax[1].dwh : ax[1].dwn;
      double v = 0, a1 = 0, a2 = 0;
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
          const double F = c < 3 ? ve[c].at(b1 + i, b2 + j, 0) : vb[c - 3].at(b1 + i, b2 + j, 0);
          v += F * w1[i] * w2[j];
          a1 += F * d1[i] * w2[j];
          a2 += F * w1[i] * d2[j];
        }
      eb[c] = v;
      g1[c] = a1 * g.inv_dx[0];
      g2[c] = a2 * g.inv_dx[1];
    }
    const Vec3 lxn = v3(A.lx[q], A.lx[A.n + q], 0.0);
    const Vec3 lu_in = v3(A.lu[q], A.lu[A.n + q], A.lu[2 * A.n + q]);
    double leb[6];
    double ldx[2] = {0.0, 0.0};   // deposit's share of the x^n adjoint
    Vec3 lum;
    if constexpr (PUSH == PIC_ANALYTIC) {
      // analytic push: its Jacobian by dual numbers through the smooth form
      const double u0[3] = {A.u[q], A.u[A.n + q], A.u[2 * A.n + q]};
      double uo[3], jac[3][9];
      analytic_push_jacobian(A.qm, g.dt, eb, u0, uo, jac);
      const Vec3 un = v3(uo[0], uo[1], uo[2]);
      const double gn = sqrt(1.0 + dot(un, un));
      const Vec3 lun = lu_in + (g.dt / gn) * (lxn - (dot(un, lxn) / (gn * gn)) * un) +
                       deposit_adjoint(A, q, g, un, gn, ldx);
      double lk[9];
      for (int k = 0; k < 9; ++k) lk[k] = lun.x * jac[0][k] + lun.y * jac[1][k] + lun.z * jac[2][k];
      lum = v3(lk[0], lk[1], lk[2]);
      for (int c = 0; c < 6; ++c) leb[c] = lk[3 + c];
    } else {
    // forward Boris with intermediates
    const double h = 0.5 * A.qm * g.dt;
    const Vec3 E = v3(eb[0], eb[1], eb[2]), B = v3(eb[3], eb[4], eb[5]);
    const Vec3 u = v3(A.u[q], A.u[A.n + q], A.u[2 * A.n + q]);
    const Vec3 um = u + h * E;
    const double ig = 1.0 / sqrt(1.0 + dot(um, um));
    const double hig = h * ig;
    const Vec3 t = hig * B;
    const double tt = dot(t, t);
    const double f = 2.0 / (1.0 + tt);
    const Vec3 sv = f * t;
    const Vec3 p = um + cross(um, t);
    const Vec3 up = um + cross(p, sv);
    const Vec3 un = up + h * E;
    const double gn = sqrt(1.0 + dot(un, un));
    // reverse
    // x^{n+1} = x^n + dt un/gn:  d(un/gn)/dun = (I - un un^T/gn^2)/gn
    const Vec3 lun = lu_in + (g.dt / gn) * (lxn - (dot(un, lxn) / (gn * gn)) * un) +
                     deposit_adjoint(A, q, g, un, gn, ldx);
    Vec3 lE = h * lun;
    const Vec3 lup = lun;
    lum = lup;
    const Vec3 lp = cross(sv, lup);
    const Vec3 ls = cross(lup, p);
    const double lf = dot(ls, t);
    Vec3 lt = f * ls;
    const double ltt = lf * (-0.5 * f * f);
    lt = lt + (2.0 * ltt) * t;
    lum = lum + lp + cross(t, lp);
    lt = lt + cross(lp, um);
    const Vec3 lB = hig * lt;
    const double lhig = dot(lt, B);
    lum = lum - (h * lhig * ig * ig * ig) * um;
    lE = lE + h * lum;
    leb[0] = lE.x; leb[1] = lE.y; leb[2] = lE.z;
    leb[3] = lB.x; leb[4] = lB.y; leb[5] = lB.z;
    }
    // position adjoint: identity from x^{n+1} = x^n + ..., plus the field gradient
    double lx1 = lxn.x + ldx[0], lx2 = lxn.y + ldx[1];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      lx1 += leb[c] * g1[c];
      lx2 += leb[c] * g2[c];
    }
    A.lu[q] = lum.x;
    A.lu[A.n + q] = lum.y;
    A.lu[2 * A.n + q] = lum.z;
    A.lx[q] = lx1;
    A.lx[A.n + q] = lx2;
    // transpose of the gather: scatter with the same weights
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int b1 = half[c][0] ? ax[0].bh : ax[0].bn;
      const int b2 = half[c][1] ? ax[1].bh : ax[1].bn;
      const double* w1 = half[c][0] ? ax[0].wh : ax[0].wn;
      const double* w2 = half[c][1] ? ax[1].wh : ax[1].wn;
      double* dst = c < 3 ? A.lE[c] : A.SB[c - 3];
      for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i)
          atomicAdd(&dst[(int64_t)wrap_index(b2 + j, n2) * n1 + wrap_index(b1 + i, n1)],
                    leb[c] * w1[i] * w2[j]);
    }
  }
}

// E += alpha * K_B[c] S  (Ampere-form curl, d^B stencil with coefficients pre-scaled
// in s.kE, i.e. dt C^E / dx1; alpha carries the remaining factor)
__global__ void curl_b_axpy_kernel(double* E0, double* E1, double* E2, const double* S0,
                                   const double* S1, const double* S2, GridArgs g,
                                   StencilArgs<double> s, double alpha) {
  const int n1 = g.n[0], n2 = g.n[1];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1), j = (int)(q / n1);
    auto at = [&](const double* a, int di, int dj) {
      return a[(int64_t)wrap_index(j + dj, n2) * n1 + wrap_index(i + di, n1)];
    };
    double dS2 = 0, dS3 = 0;
    for (int m = 1; m <= s.M; ++m) {
      dS3 += s.kE[m - 1] * (at(S2, m - 1, 0) - at(S2, -m, 0));
      dS2 += s.kE[m - 1] * (at(S1, m - 1, 0) - at(S1, -m, 0));
    }
    const double y2 = s.y2;
    E0[q] += alpha * (y2 * (at(S2, 0, 0) - at(S2, 0, -1)));
    E1[q] += alpha * (-dS3);
    E2[q] += alpha * (dS2 - y2 * (at(S0, 0, 0) - at(S0, 0, -1)));
  }
}

// m_B -= S; S = 0
__global__ void sub_clear_kernel(double* m0, double* m1, double* m2, double* S0, double* S1,
                                 double* S2, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    m0[q] -= S0[q];
    m1[q] -= S1[q];
    m2[q] -= S2[q];
    S0[q] = S1[q] = S2[q] = 0.0;
  }
}

// out += sum a*b (warp shuffles, one atomic per warp)
__global__ void dot_kernel(const double* a, const double* b, int64_t n, double* out) {
  double acc = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    acc += a[q] * b[q];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void diff_kernel(double* d, const double* a, const double* b, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    d[q] = a[q] - b[q];
}

// l_u = (1/n) u / gamma  (adjoint of the mean energy), l_x = 0
__global__ void energy_seed_kernel(const double* u, double* lu, double* lx, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double a = u[q], b = u[n + q], c = u[2 * n + q];
    const double gi = 1.0 / sqrt(1.0 + a * a + b * b + c * c);
    lu[q] = a * gi / n;
    lu[n + q] = b * gi / n;
    lu[2 * n + q] = c * gi / n;
    lx[q] = 0.0;
    lx[n + q] = 0.0;
  }
}

__global__ void energy_sum_kernel(const double* u, int64_t n, double* out) {
  double acc = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double a = u[q], b = u[n + q], c = u[2 * n + q];
    acc += sqrt(1.0 + a * a + b * b + c * c) - 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc / n);
}

// Stencil-coefficient gradient contributions of one step (x1 taps only):
//  gcE[j] += sum [ lB2 * Dj E3 - lB3 * Dj E2 ]          Dj f = f_{i+j} - f_{i-j+1}
//  gcB[j] += sum [ lE3 * DBj B2 - lE2 * DBj B3 ]        DBj f = f_{i+j-1} - f_{i-j}
// (the caller multiplies by dt/dx1 and the adjoint sign conventions)
template <int MMAX>
__global__ void coeff_grad_kernel(const double* la, const double* lb, const double* fa,
                                  const double* fb, GridArgs g, int M, int ampere, double* out) {
  const int n1 = g.n[0];
  double acc[MMAX];
#pragma unroll
  for (int m = 0; m < MMAX; ++m) acc[m] = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < g.ncell;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % n1);
    const int64_t row = q - i;
    const double A = la[q], Bv = lb[q];
#pragma unroll
    for (int m = 1; m <= MMAX; ++m) {
      if (m > M) break;
      const int ip = ampere ? i + m - 1 : i + m;
      const int im = ampere ? i - m : i - m + 1;
      const double da = fa[row + wrap_index(ip, n1)] - fa[row + wrap_index(im, n1)];
      const double db = fb[row + wrap_index(ip, n1)] - fb[row + wrap_index(im, n1)];
      acc[m - 1] += A * da - Bv * db;
    }
  }
#pragma unroll
  for (int m = 0; m < MMAX; ++m) {
    if (m >= M) break;
    double v = acc[m];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[m], v);
  }
}

inline int nblk(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

#define ACK(c, call)                                                                  \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      (c)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return e_ == cudaErrorMemoryAllocation ? PIC_ERR_OOM : PIC_ERR_CUDA;            \
    }                                                                                 \
  } while (0)

#define PCK(call)                     \
  do {                                \
    pic_status s_ = (call);           \
    if (s_ != PIC_OK) return s_;      \
  } while (0)

// device buffers owned by one adjoint call
struct Pool {
  std::vector<void*> p;
  ~Pool() {
    for (void* q : p) cudaFree(q);
  }
  cudaError_t get(double** out, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(double) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) {
      p.push_back(q);
      *out = (double*)q;
    }
    return e;
  }
};

// copy the context's current E, B into dst[6] (device)
pic_status save_fields(pic_ctx* c, double* const* dst) {
  for (int k = 0; k < 3; ++k) {
    ACK(c, cudaMemcpyAsync(dst[k], c->fe[c->cur][k], sizeof(double) * c->g.ncell,
                           cudaMemcpyDeviceToDevice, c->stream));
    ACK(c, cudaMemcpyAsync(dst[3 + k], c->fb[c->cur][k], sizeof(double) * c->g.ncell,
                           cudaMemcpyDeviceToDevice, c->stream));
  }
  return PIC_OK;
}

pic_status load_fields(pic_ctx* c, double* const* src) {
  for (int k = 0; k < 6; ++k) PCK(pic_load_field(c, k, src[k], 1));
  return PIC_OK;
}

StencilArgs<double> swapped(const pic_ctx* c) {
  StencilArgs<double> s = c->sd;
  for (int j = 0; j < PIC_MAX_M; ++j) std::swap(s.kE[j], s.kB[j]);
  return s;
}

}  // namespace

namespace {

// Laser-energy objective and its a0 / phase gradients for n particles of host
// weights w (null: test particles, weight 0).
pic_status laser_energy_adjoint(pic_ctx* c, const pic_laser* laser, int64_t n, const double* x,
                                const double* u, const double* w, int64_t nsteps, int ckp,
                                double* J, double* dJ_da0, double* dJ_dphase) {
  if (!c || !laser || n < 1 || !x || !u || nsteps < 1 || ckp < 1 || !J || !dJ_da0 || !dJ_dphase)
    return PIC_ERR_ARG;
  if (c->grid.precision != PIC_FP64 ||
      (c->grid.pusher != PIC_BORIS && c->grid.pusher != PIC_ANALYTIC) || c->grid.ndim != 2) {
    c->err = "adjoint needs a 2D PIC_FP64 context with the Boris or the analytic pusher";
    return PIC_ERR_STATE;
  }
  if (!(laser->a0 != 0.0)) {
    c->err = "a0 must be non-zero";
    return PIC_ERR_ARG;
  }
  ACK(c, cudaSetDevice(c->device));
  const int64_t nc = c->g.ncell;
  const int nseg = (int)((nsteps + ckp - 1) / ckp);
  const int seg = (int)std::min<int64_t>(ckp, nsteps);
  Pool P;
  double *F0[6], *F0p[6], *lamE[2][3], *muB[2][3], *SB[3];
  for (int k = 0; k < 6; ++k) {
    ACK(c, P.get(&F0[k], nc));
    ACK(c, P.get(&F0p[k], nc));
  }
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      ACK(c, P.get(&lamE[s][k], nc));
      ACK(c, P.get(&muB[s][k], nc));
    }
  for (int k = 0; k < 3; ++k) ACK(c, P.get(&SB[k], nc));
  std::vector<double*> ckf((size_t)nseg * 6), ckx(nseg), cku(nseg);
  for (int s = 0; s < nseg; ++s) {
    for (int k = 0; k < 6; ++k) ACK(c, P.get(&ckf[(size_t)s * 6 + k], nc));
    ACK(c, P.get(&ckx[s], 2 * n));
    ACK(c, P.get(&cku[s], 3 * n));
  }
  double *segF, *segx, *segu, *lu, *lx, *wz, *acc, *uend, *xend, *finF[6];
  ACK(c, P.get(&segF, (size_t)seg * 6 * nc));
  ACK(c, P.get(&segx, (size_t)seg * 2 * n));
  ACK(c, P.get(&segu, (size_t)seg * 3 * n));
  ACK(c, P.get(&lu, 3 * n));
  ACK(c, P.get(&lx, 2 * n));
  ACK(c, P.get(&wz, n));
  ACK(c, P.get(&acc, 4));
  ACK(c, P.get(&uend, 3 * n));
  ACK(c, P.get(&xend, 2 * n));
  for (int k = 0; k < 6; ++k) ACK(c, P.get(&finF[k], nc));
  cudaStream_t st = c->stream;
  ACK(c, cudaMemsetAsync(wz, 0, sizeof(double) * n, st));
  // weights on the device (the segment recomputations load from device arrays)
  bool has_w = false;
  if (w)
    for (int64_t q = 0; q < n && !has_w; ++q) has_w = w[q] != 0.0;
  double* wdev = wz;
  double *tmpJ1 = nullptr, *taps_rev = nullptr;
  int lo_rev = 0;
  if (has_w) {
    ACK(c, P.get(&wdev, n));
    ACK(c, cudaMemcpyAsync(wdev, w, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    if (c->corr) {
      // P^T of the x1 correction: the convolution with the reversed taps
      std::vector<double> t(c->taps_n);
      ACK(c, cudaMemcpy(t.data(), c->taps, sizeof(double) * c->taps_n, cudaMemcpyDeviceToHost));
      std::reverse(t.begin(), t.end());
      ACK(c, P.get(&taps_rev, c->taps_n));
      ACK(c, cudaMemcpy(taps_rev, t.data(), sizeof(double) * c->taps_n, cudaMemcpyHostToDevice));
      lo_rev = -(c->taps_lo + c->taps_n - 1);
      ACK(c, P.get(&tmpJ1, nc));
    }
  }
  // F0' (phase + pi/2) = dF0/dphase, then F0 itself (the initial state)
  pic_laser lp = *laser;
  lp.phase += 0.5 * M_PI;
  PCK(pic_load_laser(c, &lp));
  PCK(save_fields(c, F0p));
  PCK(pic_load_laser(c, laser));
  PCK(save_fields(c, F0));
  // the particles (host x, u, w; weight 0 when w is null)
  {
    std::vector<double> w0(n, 0.0);
    PCK(pic_load_particles(c, n, x, u, w ? w : w0.data(), -1.0, 0));
  }
  const double qm = c->qm;
  // forward with checkpoints
  for (int s = 0; s < nseg; ++s) {
    PCK(save_fields(c, &ckf[(size_t)s * 6]));
    PCK(pic_read_particles(c, ckx[s], cku[s], nullptr, 1));
    PCK(pic_step(c, std::min<int64_t>(ckp, nsteps - (int64_t)s * ckp)));
  }
  PCK(pic_read_particles(c, xend, uend, nullptr, 1));
  PCK(save_fields(c, finF));
  ACK(c, cudaMemsetAsync(acc, 0, sizeof(double) * 4, st));
  energy_sum_kernel<<<nblk(n), 256, 0, st>>>(uend, n, acc);
  energy_seed_kernel<<<nblk(n), 256, 0, st>>>(uend, lu, lx, n);
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      ACK(c, cudaMemsetAsync(lamE[s][k], 0, sizeof(double) * nc, st));
      ACK(c, cudaMemsetAsync(muB[s][k], 0, sizeof(double) * nc, st));
    }
  for (int k = 0; k < 3; ++k) ACK(c, cudaMemsetAsync(SB[k], 0, sizeof(double) * nc, st));
  const StencilArgs<double> sw = swapped(c);
  int a = 0;  // adjoint buffer parity
  for (int s = nseg - 1; s >= 0; --s) {
    const int64_t n0 = (int64_t)s * ckp, n1 = std::min<int64_t>(nsteps, n0 + ckp);
    PCK(load_fields(c, &ckf[(size_t)s * 6]));
    PCK(pic_load_particles(c, n, ckx[s], cku[s], wdev, qm, 1));
    for (int64_t k = n0; k < n1; ++k) {
      double* dst[6];
      for (int m = 0; m < 6; ++m) dst[m] = segF + ((size_t)(k - n0) * 6 + m) * nc;
      PCK(save_fields(c, dst));
      PCK(pic_read_particles(c, segx + (size_t)(k - n0) * 2 * n, segu + (size_t)(k - n0) * 3 * n,
                             nullptr, 1));
      PCK(pic_step(c, 1));
    }
    // the transposed field step below runs with no current
    for (int m = 0; m < 3; ++m)
      ACK(c, cudaMemsetAsync(c->fj[m], 0, sizeof(double) * nc, st));
    for (int64_t k = n1 - 1; k >= n0; --k) {
      // fields: l^k = A^T l^{k+1}
      FieldPtrs<double> fi, fo;
      for (int m = 0; m < 3; ++m) {
        fi.e[m] = lamE[a][m];
        fi.b[m] = muB[a][m];
        fi.j[m] = (double*)c->fj[m];  // zero (cleared above)
        fo.e[m] = lamE[1 - a][m];
        fo.b[m] = muB[1 - a][m];
        fo.j[m] = (double*)c->fj[m];
      }
      ACK(c, launch_field_step<double>(fi, fo, c->g, sw, c->ftile, c->bins.err, st));
      a = 1 - a;
      // particles at step k
      AdjPart A;
      for (int m = 0; m < 6; ++m) A.F[m] = segF + ((size_t)(k - n0) * 6 + m) * nc;
      A.x = segx + (size_t)(k - n0) * 2 * n;
      A.u = segu + (size_t)(k - n0) * 3 * n;
      A.lu = lu;
      A.lx = lx;
      for (int m = 0; m < 3; ++m) {
        A.lE[m] = lamE[a][m];
        A.SB[m] = SB[m];
      }
      A.n = n;
      A.qm = qm;
      A.pusher = c->grid.pusher;
      // current adjoint from lambda_E^{k+1} (the field step's input buffer)
      A.w = has_w ? wdev : nullptr;
      A.jscale = -c->g.dt;
      for (int m = 0; m < 3; ++m) A.lJ[m] = lamE[1 - a][m];
      if (has_w && c->corr) {
        ACK(c, cudaMemcpyAsync(tmpJ1, lamE[1 - a][0], sizeof(double) * nc, cudaMemcpyDeviceToDevice,
                               st));
        ACK(c, launch_correct_j1<double>(tmpJ1, (double*)c->jtmp, c->g, taps_rev, lo_rev,
                                         c->taps_n, c->corr_path, st));
        A.lJ[0] = tmpJ1;
      }
      if (A.pusher == PIC_ANALYTIC)
        adjoint_particle_kernel<PIC_ANALYTIC><<<nblk(n), 128, 0, st>>>(A, c->g, c->sd);
      else
        adjoint_particle_kernel<PIC_BORIS><<<nblk(n), 128, 0, st>>>(A, c->g, c->sd);
      // time-centred B: l_B += S, l_E += -(1/2) K_B[C^E] S  (m_B = -l_B)
      curl_b_axpy_kernel<<<nblk(nc), 256, 0, st>>>(lamE[a][0], lamE[a][1], lamE[a][2], SB[0],
                                                   SB[1], SB[2], c->g, c->sd, -0.5);
      sub_clear_kernel<<<nblk(nc), 256, 0, st>>>(muB[a][0], muB[a][1], muB[a][2], SB[0], SB[1],
                                                 SB[2], nc);
      ACK(c, cudaGetLastError());
    }
  }
  // gradients: <l_E, dE0> + <l_B, dB0> = <l_E, dE0> - <m_B, dB0>
  for (int k = 0; k < 3; ++k) {
    dot_kernel<<<nblk(nc), 256, 0, st>>>(lamE[a][k], F0[k], nc, acc + 1);
    dot_kernel<<<nblk(nc), 256, 0, st>>>(lamE[a][k], F0p[k], nc, acc + 2);
    dot_kernel<<<nblk(nc), 256, 0, st>>>(muB[a][k], F0[3 + k], nc, acc + 3);
  }
  double h[4];
  ACK(c, cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, st));
  ACK(c, cudaStreamSynchronize(st));
  double mB_F0p = 0;
  {
    double* acc2;
    ACK(c, P.get(&acc2, 1));
    ACK(c, cudaMemsetAsync(acc2, 0, sizeof(double), st));
    for (int k = 0; k < 3; ++k) dot_kernel<<<nblk(nc), 256, 0, st>>>(muB[a][k], F0p[3 + k], nc, acc2);
    ACK(c, cudaMemcpyAsync(&mB_F0p, acc2, sizeof(double), cudaMemcpyDeviceToHost, st));
    ACK(c, cudaStreamSynchronize(st));
  }
  *J = h[0];
  *dJ_da0 = (h[1] - h[3]) / laser->a0;
  *dJ_dphase = h[2] - mB_F0p;
  // leave the state at the end of the forward run
  PCK(load_fields(c, finF));
  PCK(pic_load_particles(c, n, xend, uend, wdev, qm, 1));
  return pic_sync(c);
}

}  // namespace

extern "C" pic_status pic_adjoint_laser_energy(pic_ctx* c, const pic_laser* laser, int64_t n,
                                               const double* x, const double* u, int64_t nsteps,
                                               int ckp, double* J, double* dJ_da0,
                                               double* dJ_dphase) {
  return laser_energy_adjoint(c, laser, n, x, u, nullptr, nsteps, ckp, J, dJ_da0, dJ_dphase);
}

extern "C" pic_status pic_adjoint_laser_energy_w(pic_ctx* c, const pic_laser* laser, int64_t n,
                                                 const double* x, const double* u, const double* w,
                                                 int64_t nsteps, int ckp, double* J,
                                                 double* dJ_da0, double* dJ_dphase) {
  if (!w) return PIC_ERR_ARG;
  return laser_energy_adjoint(c, laser, n, x, u, w, nsteps, ckp, J, dJ_da0, dJ_dphase);
}

extern "C" pic_status pic_adjoint_dispersion(pic_ctx* c, const double* e2_0, const double* b3_0,
                                             const double* target, int64_t nsteps, int ckp,
                                             double* J, double* dJ_dcE, double* dJ_dcB) {
  if (!c || !e2_0 || !b3_0 || !target || nsteps < 1 || ckp < 1 || !J || !dJ_dcE || !dJ_dcB)
    return PIC_ERR_ARG;
  if (c->grid.precision != PIC_FP64) {
    c->err = "adjoint needs a PIC_FP64 context";
    return PIC_ERR_STATE;
  }
  ACK(c, cudaSetDevice(c->device));
  const int64_t nc = c->g.ncell;
  const int M = c->M;
  const int nseg = (int)((nsteps + ckp - 1) / ckp);
  const int seg = (int)std::min<int64_t>(ckp, nsteps);
  cudaStream_t st = c->stream;
  Pool P;
  double *lamE[2][3], *muB[2][3], *tgt, *acc, *gE, *gB, *finF[6];
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      ACK(c, P.get(&lamE[s][k], nc));
      ACK(c, P.get(&muB[s][k], nc));
    }
  ACK(c, P.get(&tgt, nc));
  ACK(c, P.get(&acc, 1));
  ACK(c, P.get(&gE, PIC_MAX_M));
  ACK(c, P.get(&gB, PIC_MAX_M));
  for (int k = 0; k < 6; ++k) ACK(c, P.get(&finF[k], nc));
  std::vector<double*> ckf((size_t)nseg * 6);
  for (auto& p : ckf) ACK(c, P.get(&p, nc));
  double* segF;
  ACK(c, P.get(&segF, (size_t)(seg + 1) * 6 * nc));
  ACK(c, cudaMemcpyAsync(tgt, target, sizeof(double) * nc, cudaMemcpyHostToDevice, st));
  // initial state: E2, B3 given, the rest zero, no particles
  {
    std::vector<double> z(nc, 0.0);
    for (int k = 0; k < 6; ++k)
      PCK(pic_load_field(c, k, k == PIC_E2 ? e2_0 : (k == PIC_B3 ? b3_0 : z.data()), 0));
    PCK(pic_load_particles(c, 0, nullptr, nullptr, nullptr, -1.0, 0));
  }
  for (int s = 0; s < nseg; ++s) {
    PCK(save_fields(c, &ckf[(size_t)s * 6]));
    PCK(pic_step(c, std::min<int64_t>(ckp, nsteps - (int64_t)s * ckp)));
  }
  PCK(save_fields(c, finF));
  // J = 1/2 |E2^N - target|^2;  seed l_E2 = E2^N - target
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      ACK(c, cudaMemsetAsync(lamE[s][k], 0, sizeof(double) * nc, st));
      ACK(c, cudaMemsetAsync(muB[s][k], 0, sizeof(double) * nc, st));
    }
  diff_kernel<<<nblk(nc), 256, 0, st>>>(lamE[0][1], finF[1], tgt, nc);
  ACK(c, cudaMemsetAsync(acc, 0, sizeof(double), st));
  dot_kernel<<<nblk(nc), 256, 0, st>>>(lamE[0][1], lamE[0][1], nc, acc);
  ACK(c, cudaMemsetAsync(gE, 0, sizeof(double) * PIC_MAX_M, st));
  ACK(c, cudaMemsetAsync(gB, 0, sizeof(double) * PIC_MAX_M, st));
  const StencilArgs<double> sw = swapped(c);
  int a = 0;
  for (int s = nseg - 1; s >= 0; --s) {
    const int64_t n0 = (int64_t)s * ckp, n1 = std::min<int64_t>(nsteps, n0 + ckp);
    PCK(load_fields(c, &ckf[(size_t)s * 6]));
    for (int64_t k = n0; k <= n1; ++k) {
      double* dst[6];
      for (int m = 0; m < 6; ++m) dst[m] = segF + ((size_t)(k - n0) * 6 + m) * nc;
      PCK(save_fields(c, dst));
      if (k < n1) PCK(pic_step(c, 1));
    }
    for (int64_t k = n1 - 1; k >= n0; --k) {
      const double* Fk = segF + (size_t)(k - n0) * 6 * nc;        // E^k, B^{k-1/2}
      const double* Fk1 = segF + (size_t)(k + 1 - n0) * 6 * nc;   // E^{k+1}, B^{k+1/2}
      // dJ/dC^B: <l_E^{k+1}, dE^{k+1}/dC^B> with B^{k+1/2}:  l_E3 DB B2 - l_E2 DB B3
      coeff_grad_kernel<PIC_MAX_M><<<nblk(nc), 256, 0, st>>>(
          lamE[a][2], lamE[a][1], Fk1 + 4 * nc, Fk1 + 5 * nc, c->g, M, 1, gB);
      FieldPtrs<double> fi, fo;
      for (int m = 0; m < 3; ++m) {
        fi.e[m] = lamE[a][m];
        fi.b[m] = muB[a][m];
        fi.j[m] = (double*)c->fj[m];
        fo.e[m] = lamE[1 - a][m];
        fo.b[m] = muB[1 - a][m];
        fo.j[m] = (double*)c->fj[m];
      }
      ACK(c, launch_field_step<double>(fi, fo, c->g, sw, c->ftile, c->bins.err, st));
      a = 1 - a;
      // dJ/dC^E: <l_B'', dB'/dC^E> with l_B'' = -m_B^k:  l_B2 D E3 - l_B3 D E2
      //        = (-m_B3) ... written as  m_B3 D E2 - m_B2 D E3
      coeff_grad_kernel<PIC_MAX_M><<<nblk(nc), 256, 0, st>>>(
          muB[a][2], muB[a][1], Fk + 1 * nc, Fk + 2 * nc, c->g, M, 0, gE);
      ACK(c, cudaGetLastError());
    }
  }
  double hJ = 0, hE[PIC_MAX_M], hB[PIC_MAX_M];
  ACK(c, cudaMemcpyAsync(&hJ, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  ACK(c, cudaMemcpyAsync(hE, gE, sizeof(double) * M, cudaMemcpyDeviceToHost, st));
  ACK(c, cudaMemcpyAsync(hB, gB, sizeof(double) * M, cudaMemcpyDeviceToHost, st));
  ACK(c, cudaStreamSynchronize(st));
  const double scale = c->dt / c->g.dx[0];
  *J = 0.5 * hJ;
  for (int j = 0; j < M; ++j) {
    dJ_dcE[j] = scale * hE[j];
    dJ_dcB[j] = scale * hB[j];
  }
  PCK(load_fields(c, finF));
  return pic_sync(c);
}

// Host copy of the analytic push's vector-Jacobian product (analytic_vjp.cuh),
// for checking the derivative code without a device.
extern "C" pic_status pic_analytic_push_vjp(double qm, double dt, const double* eb,
                                            const double* u, const double* lam, double* u_out,
                                            double* d_eb, double* d_u) {
  if (!eb || !u || !lam || !u_out || !d_eb || !d_u || !(dt > 0)) return PIC_ERR_ARG;
  double jac[3][9];
  const bool ok = pic::analytic_push_jacobian(qm, dt, eb, u, u_out, jac);
  for (int k = 0; k < 9; ++k) {
    const double v = lam[0] * jac[0][k] + lam[1] * jac[1][k] + lam[2] * jac[2][k];
    if (k < 3) d_u[k] = v;
    else d_eb[k - 3] = v;
  }
  return ok ? PIC_OK : PIC_ERR_DEVICE_CHECK;
}
