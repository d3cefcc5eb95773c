/*
 * pic.h -- C ABI of libpic, a single-GPU (GB300, sm_103a) electromagnetic
 * particle-in-cell time step built around the customised dual-stencil field
 * solver of Li et al., "A new field solver for modeling of relativistic
 * particle-laser interactions using the particle-in-cell algorithm"
 * (arXiv:2004.03754).
 *
 * Physics (normalised units c = m_e = e = 1, Sec. 2.1):
 *   Faraday  B^{n+1/2} = B^{n-1/2} - dt  d_E x E^n            (Eq. (1))
 *   Ampere   E^{n+1}   = E^n + dt (d_B x B^{n+1/2} - J^{n+1/2}) (Eq. (1))
 *   x1 derivatives use M-coefficient stencils, different in the two laws:
 *     d^E f_i = (1/dx1) sum_j C^E_j (f_{i+j} - f_{i-j+1})      (App. B Eq. (B.1))
 *     d^B f_i = (1/dx1) sum_j C^B_j (f_{i+j-1} - f_{i-j})      (App. B Eq. (B.2))
 *   x2, x3 derivatives are Yee (Sec. 3.1.1).  Particles see E^n and the
 *   time-centred B^n = (B^{n-1/2}+B^{n+1/2})/2 (Eq. (7)) through a quadratic
 *   B-spline at each component's staggered node (App. A), are pushed by the
 *   Boris or the analytic constant-field pusher (Sec. 1, Sec. 4.1), move by
 *   x^{n+1} = x^n + dt u/gamma, and deposit an Esirkepov charge-conserving
 *   current (Sec. 3.3), corrected along x1 by ([k]_Yee/[k]_B1) so that Gauss's
 *   law holds with d_B (Sec. 3.3, Eqs. (23)-(26)).
 *
 * Layout: every field component is an array of n1*n2*n3 values, x1 fastest,
 * idx = (k*n2 + j)*n1 + i; Yee staggering E1(i+1/2,j,k) E2(i,j+1/2,k)
 * E3(i,j,k+1/2) B1(i,j+1/2,k+1/2) B2(i+1/2,j,k+1/2) B3(i+1/2,j+1/2,k); J is
 * co-located with E.  In 2D n3 = 1 and the x3 offsets drop out.  All axes are
 * periodic.  Particle arrays are structure-of-arrays: x[d*n + p] (d < ndim),
 * u[c*n + p] (c < 3, u = gamma*beta), w[p] (charge density carried by the
 * particle when its shape sums to one; 0 marks a test particle that is pushed
 * but never deposits).
 *
 * Ownership and errors: the context owns all device memory it allocates; input
 * buffers are copied, output buffers belong to the caller.  Every call returns
 * a pic_status and none aborts.  Device-side checks latch an error word that
 * the next synchronising call (pic_sync, pic_read_*) returns as
 * PIC_ERR_DEVICE_CHECK; pic_last_error() gives a one-line description.  All
 * work is issued on the stream given to pic_init (0 = legacy default stream).
 * A context is not thread-safe.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
  PIC_OK = 0,
  PIC_ERR_ARG = -1,          /* invalid argument (null pointer, size, enum) */
  PIC_ERR_CFL = -2,          /* dt violates the CFL condition of Eq. (21) */
  PIC_ERR_OOM = -3,          /* device allocation failed */
  PIC_ERR_CUDA = -4,         /* a CUDA runtime call failed */
  PIC_ERR_DEVICE_CHECK = -5, /* a device-side check failed (see pic_last_error) */
  PIC_ERR_TIMEOUT = -6,      /* a bounded device-side wait ran out */
  PIC_ERR_STATE = -7         /* call not valid in the context's current state */
} pic_status;

/* precision:
 *   PIC_FP64         every field and particle quantity in FP64;
 *   PIC_MIXED        fields, gather and deposit in FP32, momentum/gamma/positions FP64
 *                    (field error ~6e-8 relative per value; the single-electron
 *                    energy leaves 1e-4 of FP64 beyond a0 ~ 10, see below);
 *   PIC_COMPENSATED  E and B stored and updated as FP32 pairs hi + lo (48-bit
 *                    significand, FP32 error-free arithmetic, 8 bytes per value),
 *                    gather in that arithmetic, push and positions FP64, current
 *                    accumulated in FP32.  An electron co-moving with a laser feels
 *                    E2 - beta1 B3 ~ E/(2 gamma^2) (Sec. 1), so FP32 field rounding is
 *                    amplified by ~gamma^2; the compensated fields keep the
 *                    single-electron energy within 1e-4 of FP64 up to a0 = 1e4. */
enum { PIC_FP64 = 0, PIC_MIXED = 1, PIC_COMPENSATED = 2 };
/* particle pusher: Boris (Sec. 1), analytic for constant fields over a step
 * (Sec. 1, Sec. 4.1), Higuera-Cary (Sec. 1, Sec. 4.1; Higuera & Cary 2017) */
enum { PIC_BORIS = 0, PIC_ANALYTIC = 1, PIC_HC = 2 };

/* Field component selectors for pic_load_field / pic_read_field. */
enum {
  PIC_E1 = 0, PIC_E2 = 1, PIC_E3 = 2,
  PIC_B1 = 3, PIC_B2 = 4, PIC_B3 = 5,       /* B^{n-1/2}: the leapfrog state */
  PIC_J1 = 6, PIC_J2 = 7, PIC_J3 = 8,       /* current used by the last step (after
                                               the x1 correction) */
  PIC_BBAR1 = 9, PIC_BBAR2 = 10, PIC_BBAR3 = 11 /* time-centred B^n (read only) */
};

typedef struct {
  int ndim;          /* 2 (2D3V) or 3 */
  int n[3];          /* cells per axis; n[2] ignored (taken as 1) in 2D */
  double dx[3];      /* cell sizes; dx[2] ignored in 2D */
  int precision;     /* PIC_FP64, PIC_MIXED or PIC_COMPENSATED */
  int pusher;        /* PIC_BORIS, PIC_ANALYTIC or PIC_HC */
  int shape;         /* particle shape order: 0 or PIC_SHAPE_QUADRATIC (the quadratic
                        B-spline of App. A, the only one built); other values PIC_ERR_ARG */
  int boundary;      /* 0 or PIC_BOUNDARY_PERIODIC (periodic on every axis, the only one
                        built; the moving window of pic_set_moving_window shifts along x1
                        on top of it); other values PIC_ERR_ARG */
} pic_grid;

#define PIC_SHAPE_QUADRATIC 2
#define PIC_BOUNDARY_PERIODIC 1

typedef struct {
  int M;             /* number of x1 coefficients, 1 <= M <= PIC_MAX_M */
  const double* cE;  /* C^E_1..C^E_M (Faraday), App. B Eq. (B.1) */
  const double* cB;  /* C^B_1..C^B_M (Ampere),  App. B Eq. (B.2) */
} pic_coeffs;

#define PIC_MAX_M 32

typedef struct {
  double a0;         /* peak normalised vector potential eA/mc^2 (Sec. 1) */
  double k0;         /* laser wavenumber */
  double phase;      /* carrier phase */
  double L_env;      /* sin^2 envelope length; must not exceed n1*dx1 */
  double x_front;    /* leading edge position along x1 at t = 0 */
  double w0;         /* Gaussian transverse waist (field e^-r^2/w0^2); <= 0: plane wave */
  double x2c, x3c;   /* transverse centre */
} pic_laser;

typedef struct {
  int sort_interval;       /* steps between particle re-binning */
  int tile[3];             /* particle tile (cells) */
  int guard[3];            /* staging guard of the particle kernel: cells above the
                              tile (one fewer below) */
  int64_t n_particles;
  int64_t steps_done;
  int64_t last_stragglers; /* particles of the last step that fell outside their
                              tile's staged window and took the global path */
  int correction_active;   /* 1 when C^B != e_1 (x1 current correction runs) */
  double cfl_lhs;          /* max over k of the left side of Eq. (21) */
  double cfl_sufficient_dt;/* bound of Eq. (22) */
  int kernels_per_step;    /* kernel launches of one pic_step(ctx, 1) */
} pic_info;

/* Create a context: validates the grid, copies the coefficients, checks the
 * exact CFL condition of Eq. (21) (max over k1 of (dt/2)^2 ([k]_B1 [k]_E1 +
 * sum_{i>1} (2/dx_i)^2) <= 1, and [k]_B1 [k]_E1 >= 0 for every k1) and
 * allocates the fields, which start at zero.  stream: a cudaStream_t or NULL.
 * Errors: PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_OOM, PIC_ERR_CUDA; *out = NULL then. */
pic_status pic_init(const pic_grid* grid, double dt, const pic_coeffs* coeffs, void* stream,
                    pic_ctx** out);

/* Load E^0 and B^{-1/2} of an x2-polarised sin^2 pulse moving in +x1, defined
 * by a(phi) = a0 sin^2(pi phi/L_env) sin(k0 phi + phase), phi = x_front - x1,
 * E2 = -da/dt, times exp(-(x2-x2c)^2/w0^2) (and x3).  B3^{-1/2} is the
 * discrete forward eigenmode partner of E2 per x1-Fourier mode, Eq. (8):
 * B3~ = ([k]_E1/[omega]_t) E2~ e^{i k dx1/2} e^{i omega dt/2}, omega from Eq. (4);
 * the Nyquist mode of B3 is zero.  All other components are set to zero.
 * Setup only (host DFT of the 1D profile, then one expansion kernel). */
pic_status pic_load_laser(pic_ctx* ctx, const pic_laser* laser);

/* Copy one component (PIC_E1..PIC_B3, the state) from an FP64 buffer of
 * n1*n2*n3 values; on_device = 1 if buf is a device pointer. */
pic_status pic_load_field(pic_ctx* ctx, int comp, const double* buf, int on_device);

/* Replace the particle set: n particles, SoA FP64 arrays laid out as above,
 * qm = charge/mass of the species (-1 for electrons).  Positions must lie in
 * [0, n_d*dx_d); they are checked on the device.  Host buffers: the call
 * synchronises and returns PIC_ERR_ARG for an out-of-box position, leaving the
 * context with no particles.  Device buffers: the call returns at once and an
 * out-of-box position is reported by the next synchronising call
 * (PIC_ERR_DEVICE_CHECK).  The particles are re-binned by tile on the device;
 * pic_read_particles returns them in the original order. */
pic_status pic_load_particles(pic_ctx* ctx, int64_t n, const double* x, const double* u,
                              const double* w, double qm, int on_device);

/* Advance nsteps full steps (Sec. 2-3 scheme): gather E^n and the time-centred
 * B^n, push u^{n-1/2} -> u^{n+1/2}, move, deposit J^{n+1/2}, correct J1 when
 * C^B != e_1, Faraday, Ampere.  Asynchronous on the context's stream.  Pairs of
 * steps between particle re-binnings are captured once into a CUDA graph (per
 * field parity and particle buffer) and replayed, unless timing is enabled;
 * the first such call therefore captures on the context's stream and should not
 * itself run inside a stream capture.  Results do not depend on it. */
pic_status pic_step(pic_ctx* ctx, int64_t nsteps);

/* Copy one field component (any selector above) into an FP64 buffer of
 * n1*n2*n3 values.  Host buffers: the call synchronises the stream.  Device
 * buffers: the copy is enqueued on the stream and the call returns at once. */
pic_status pic_read_field(pic_ctx* ctx, int comp, double* buf, int on_device);

/* Copy the particles (original order) into x (ndim*n), u (3*n) and w (n);
 * any pointer may be NULL to skip that array.  Synchronises like pic_read_field. */
pic_status pic_read_particles(pic_ctx* ctx, double* x, double* u, double* w, int on_device);

/* Energy-gain integrals of Sec. 4.2 per particle: the work done on each particle by
 * the longitudinal field, W_LWFA = (q/m) sum_n dt E1 vbar1 (= -int v1 E1 dt for
 * electrons), and by the transverse field, W_DLA = (q/m) sum_n dt E_perp . vbar_perp,
 * with E the field the push uses (E^n at x^n) and vbar = (u^{n-1/2} + u^{n+1/2}) /
 * (gamma^{n-1/2} + gamma^{n+1/2}); for the Boris pusher W_LWFA + W_DLA is exactly the
 * particle's change of gamma.  pic_set_energy_gain(ctx, 1) allocates two FP64
 * values per particle of capacity, sets them to zero and accumulates from then on
 * (every pic_load_particles restarts them at zero); 0 frees them.  Each step then
 * runs a particle-kernel instance that also carries these sums.
 * pic_read_energy_gain copies W_LWFA and W_DLA in load order into caller-owned host
 * arrays of np values each; PIC_ERR_STATE when the integrals are off. */
pic_status pic_set_energy_gain(pic_ctx* ctx, int on);

/* Moving window along x1 (Sec. 4.1 uses moving-window boundaries along x1; the
 * paper names the boundary and gives no details, so it is read as follows).  The
 * window moves at c = 1: after every step, each time c t (counted from start_step
 * further steps on) crosses another multiple of dx1, the trailing x1 column -- the
 * one at index `origin` -- becomes fresh vacuum (E, B, J set to zero there), the
 * particles whose cell is that column are removed (the others keep their load
 * order; pic_read_particles then returns the survivors), and the column becomes
 * the window's leading one (origin advances by one, modulo n1).  No field data
 * moves: window index = (i - origin) mod n1.  start_step >= 0 turns the window on
 * (steps then run one at a time, each shift re-bins the particles and reads the
 * surviving count back); start_step < 0 turns it off.  pic_get_window returns the
 * current origin and the number of shifts since the last pic_set_moving_window. */
pic_status pic_set_moving_window(pic_ctx* ctx, int64_t start_step);

/* Spectral x1 field path (Sec. 3.1: the solver is defined by its k-space operators
 * [k]_E1 (Faraday) and [k]_B1 (Ampere), Eqs. (11)-(15), which an FFT solver can use
 * directly; Sec. 4.1 notes the same for spectral solvers).  From the next step on,
 * every x1 derivative is taken in Fourier space along x1: integer -> half-integer
 * nodes by i [k]_E1 e^{+i k dx1/2}, half-integer -> integer by i [k]_B1 e^{-i k dx1/2};
 * x2/x3 stay Yee differences; the deposited J1 is multiplied by [k]_Yee/[k]_B1 per
 * x1 mode (Sec. 3.3, Eq. (23) read as in the finite-difference path; the k = 0 mode
 * by 1/slope0, slope0 = d[k]_B1/dk at k = 0, 1 for the target operators of Eq. (15)).
 * kE1, kB1: nbins = n1/2 + 1 values at k_m = 2 pi m/(n1 dx1), m = 0..n1/2, copied.
 * The time-centred B of the gather is formed from the spectral Faraday update.  FP64
 * contexts only (PIC_ERR_STATE otherwise); bad sizes or a zero [k]_B1 at k > 0 give
 * PIC_ERR_ARG.  nbins = 0 returns to the finite-difference stencils.  The transforms
 * are cuFFT batched real-to-complex / complex-to-real plans (cuFFT allocates their
 * work areas).  Steps then run one at a time. */
pic_status pic_set_spectral(pic_ctx* ctx, int nbins, const double* kE1, const double* kB1,
                            double slope0);
pic_status pic_get_window(pic_ctx* ctx, int64_t* origin, int64_t* shifts);
pic_status pic_read_energy_gain(pic_ctx* ctx, double* w_lwfa, double* w_dla);

/* Taps of the x1 current correction (Sec. 3.3, Eq. (23)) on a periodic row of n1
 * cells of width dx1 for Ampere coefficients cB[0..M-1]: the correction is the
 * periodic convolution J1'_i = sum_q taps[q] J1_{i+lo+q}, q < *count, with the
 * inverse-DFT taps of the symbol [k]_Yee/[k]_B1 cut where they fall below 1e-15
 * of its maximum (the form pic_step applies; identity taps when C^B = e_1).
 * Host-only: no device, no allocation visible to the caller.  taps must hold
 * n1 values (the most there can be); *lo and *count are written.  PIC_ERR_ARG for
 * null pointers, n1 < 1, M outside [1, PIC_MAX_M], dx1 <= 0, or a [k]_B1 that
 * vanishes at a grid mode. */
pic_status pic_correction_taps(int n1, double dx1, int M, const double* cB, double* taps,
                               int* lo, int* count);

/* The x1 profiles pic_load_laser expands over the grid (before the transverse
 * factor of w0): E2^0 at the integer x1 nodes, -da/dt of the sin^2 pulse, and
 * B3^{-1/2} at the half nodes, its discrete forward eigenmode partner per x1
 * Fourier mode (Eq. (8)), on a periodic row of n1 cells of width dx1 with time
 * step dt.  Host-only: no device.  e2 and b3 hold n1 values each (caller-owned).
 * PIC_ERR_ARG for null pointers, n1 < 1, dx1 <= 0, dt <= 0, M outside
 * [1, PIC_MAX_M], or the laser checks of pic_load_laser (envelope longer than
 * the box, k0 <= 0, non-finite a0). */
pic_status pic_laser_profile(int n1, double dx1, double dt, const pic_coeffs* coeffs,
                             const pic_laser* laser, double* e2, double* b3);

/* Checkpoint / resume.  The state of a context is E^n and B^{n-1/2} (the
 * leapfrog state of Eq. (1)), the particles (x^n, u^{n-1/2}, w, q/m) and the
 * step count; the current J and the time-centred B are rebuilt by the next
 * step.  Layout of the caller-owned host buffer: a 64-byte-aligned header
 * (magic "PICSTATE", version, grid, dt, coefficients, counts), E1 E2 E3 B1 B2 B3
 * in the field precision (n1*n2*n3 values each, x1 fastest), then the particles
 * in load order as FP64 x (ndim*n), u (3*n), w (n).  pic_state_size gives the
 * bytes the current state needs.  pic_save_state synchronises the stream and
 * returns a latched device error instead of saving; PIC_ERR_ARG when the buffer
 * is smaller than pic_state_size.  pic_load_state accepts a state saved from a
 * context with the same grid, precision, dt and coefficients (PIC_ERR_ARG
 * otherwise, or for a truncated buffer), replaces fields and particles (the
 * particles are loaded as pic_load_particles does, with its position check) and
 * the step count; stepping on reproduces the run that was saved. */
pic_status pic_state_size(pic_ctx* ctx, size_t* bytes);
pic_status pic_save_state(pic_ctx* ctx, void* buf, size_t bytes);
pic_status pic_load_state(pic_ctx* ctx, const void* buf, size_t bytes);

/* Wait for the context's stream and return a latched device-side error, if any. */
pic_status pic_sync(pic_ctx* ctx);

/* Fill *info (host struct). */
pic_status pic_get_info(pic_ctx* ctx, pic_info* info);

/* Override the particle re-binning interval (>= 1).  Correctness does not
 * depend on it: particles outside their tile's window take a global path. */
pic_status pic_set_sort_interval(pic_ctx* ctx, int interval);

/* Field tile of the fused Faraday + Ampere kernel (App. B Eqs. (B.1)-(B.2)):
 * t1 x t2 (x t3) cells, x1 fastest; 2D grids need t3 = 1; threads (128, 256 or
 * 512) per CTA.  staging = 0 lets the kernel stream rows per warp (below) or
 * tiles into shared memory with asynchronous bulk copies where the row pitch
 * allows (n1 and t1 multiples of 16 bytes) and falls back to plain loads
 * elsewhere; staging = 2 takes the asynchronous tiles but not the row streaming;
 * staging = 1 always uses plain loads.  Results do not depend on the choice.  PIC_ERR_ARG when an extent is out of range, t1 is not a
 * multiple of 16 bytes of the field type (4 values in FP32 fields, 2 in FP64) or
 * the tile's shared-memory footprint exceeds 200 KB. */
pic_status pic_set_field_tile(pic_ctx* ctx, int t1, int t2, int t3, int threads, int staging);

/* With staging 0 (and n1 a multiple of 16 bytes of the field type) fields are
 * updated row by row, streamed along x2: a work item is a strip of `width` x1
 * columns by `rows` rows (0: chosen so that the items fill the resident CTAs
 * evenly), and a ring of `stages` rows of E^n and B^{n-1/2} (and J in 3D with
 * one warp per plane; elsewhere J is read into registers) is kept in flight.  In 2D `warps` warps per CTA take items independently, each with its
 * own ring.  In 3D `warps` = 1 gives each warp one x3 plane (each stage holding
 * E at that plane and its two neighbours and B at the plane and the one below);
 * `warps` = P > 1 gives a CTA of P warps a group of P consecutive x3 planes,
 * one warp per plane, sharing one ring of the group's rows.
 * Results do not depend on the choice.  PIC_ERR_ARG when width is not a
 * positive multiple of 16 bytes of the field type, rows < 0, warps outside
 * [1, 16] (in 3D [1, 8]), stages outside [2, 8], or the rows do not fit in 200 KB
 * of shared memory. */
pic_status pic_set_field_strip(pic_ctx* ctx, int width, int rows, int warps, int stages);

/* Form of the x1 current correction (Sec. 3.3, Eq. (23)), the periodic
 * convolution of every x1 row of J1 with the taps of P^{-1}: 0 automatic (1 when
 * a row and the taps fit in 200 KB of shared memory, else 2 when the taps do,
 * else 3), 1 whole rows staged in shared memory and updated in place, 2 row
 * segments of 1024 cells out of place, 3 straight from global memory.  All forms
 * give bit-identical results.  PIC_ERR_ARG for a path outside [0, 3] or a form
 * whose shared memory does not fit this grid.  No effect when C^B = e_1. */
pic_status pic_set_correction_path(pic_ctx* ctx, int path);

/* Per-kernel device time, accumulated with CUDA events recorded on the
 * context's stream around each kernel group while timing is enabled. */
typedef struct {
  double ms_rebin;      /* particle re-binning (count, scan, scatter) */
  double ms_particles;  /* gather + push + deposit (tiled kernel) */
  double ms_stragglers; /* global-path particles */
  double ms_correction; /* x1 current correction */
  double ms_fields;     /* fused Faraday + Ampere */
  int64_t launches;     /* libpic kernels launched while timing was enabled */
  int64_t steps;        /* steps timed */
} pic_timing;

/* Enable (1) or disable (0) event timing; enabling clears the accumulators. */
pic_status pic_set_timing(pic_ctx* ctx, int enable);

/* Synchronise the stream and return the accumulated times. */
pic_status pic_get_timing(pic_ctx* ctx, pic_timing* out);

/* ------------------------------------------------------------------------
 * Adjoint (reverse mode) of the whole step, FP64 contexts.  The field step's
 * transpose is the same fused stencil update with C^E and C^B exchanged,
 * acting on (lambda_E, -lambda_B); the gather's transpose scatters with the
 * same shape weights; the Boris push is differentiated by hand, the analytic
 * push by dual numbers through its smooth form; the Esirkepov deposit of
 * depositing particles by dual numbers through the deposit itself; the forward
 * trajectory is checkpointed every `checkpoint_every` steps and each segment
 * recomputed before it is swept backwards.  The calls leave the context's
 * state at the end of the forward run.
 * ------------------------------------------------------------------------ */

/* Host-only: the analytic push (constant E, B over dt; Sec. 1, Sec. 4.1) in its
 * smooth form and its vector-Jacobian product, the same code the adjoint's particle
 * kernel runs.  eb = (E1..E3, B1..B3) at the particle, u = u^{n-1/2}, lam = the
 * adjoint of u^{n+1/2} (3 values each); writes u_out = u^{n+1/2}, d_eb[6] =
 * lam . d u_out/d eb and d_u[3] = lam . d u_out/d u.  PIC_ERR_ARG on null
 * pointers or dt <= 0; PIC_ERR_DEVICE_CHECK if the proper-time iteration did not
 * converge (outputs then unreliable).  No device is used. */
pic_status pic_analytic_push_vjp(double qm, double dt, const double* eb, const double* u,
                                 const double* lam, double* u_out, double* d_eb, double* d_u);

/* J = mean over the n test particles (weight 0) of (gamma - 1) after nsteps
 * steps (Boris or analytic pusher), starting from the laser `laser` and the particles x (ndim*n),
 * u (3*n), all host FP64.  Returns J and dJ/d(a0), dJ/d(phase).  Needs a
 * 2D PIC_FP64 context with the Boris or the analytic pusher; otherwise
 * PIC_ERR_STATE. */
pic_status pic_adjoint_laser_energy(pic_ctx* ctx, const pic_laser* laser, int64_t n,
                                    const double* x, const double* u, int64_t nsteps,
                                    int checkpoint_every, double* J, double* dJ_da0,
                                    double* dJ_dphase);

/* The same objective for n particles of host weights w (n values, FP64): those
 * of non-zero weight deposit J^{n+1/2} (Sec. 3.3, Eq. (24)) in the forward run,
 * and the reverse pass carries the current's adjoint lambda_J = -dt P^T lambda_E
 * (P: the x1 current correction, Eq. (23)) back through the deposit into each
 * particle's x^n and u^{n+1/2}.  J stays the unweighted mean of (gamma - 1).
 * Same context requirements and errors as above; PIC_ERR_ARG when w is null. */
pic_status pic_adjoint_laser_energy_w(pic_ctx* ctx, const pic_laser* laser, int64_t n,
                                      const double* x, const double* u, const double* w,
                                      int64_t nsteps, int checkpoint_every, double* J,
                                      double* dJ_da0, double* dJ_dphase);

/* Vacuum dispersion objective J = (1/2) sum_cells (E2^N - target)^2 after
 * nsteps field steps from E2^0 = e2_0, B3^{-1/2} = b3_0 (all other components
 * zero; host FP64 arrays of n1*n2*n3).  Returns J and dJ/dC^E, dJ/dC^B (M values
 * each).  Needs a PIC_FP64 context. */
pic_status pic_adjoint_dispersion(pic_ctx* ctx, const double* e2_0, const double* b3_0,
                                  const double* target, int64_t nsteps, int checkpoint_every,
                                  double* J, double* dJ_dcE, double* dJ_dcB);

/* ------------------------------------------------------------------------
 * Ensembles: many independent 2D runs of uneven grid sizes advanced together
 * by ONE persistent kernel launch (captured in a CUDA graph).  All runs share
 * dx, dt, the x1 stencil, precision and pusher; each has its own grid size,
 * laser, particles and step count.  Runs are not coupled.  The field work of
 * the persistent kernel is streamed row by row per warp over x1 strips; the
 * strip shape is chosen by pic_batch_autotune.
 * ------------------------------------------------------------------------ */
typedef struct pic_batch pic_batch;

typedef struct {
  int nruns;          /* >= 1 */
  const int* n1;      /* nruns cells along x1 */
  const int* n2;      /* nruns cells along x2 */
  double dx[2];       /* shared cell sizes */
  int precision;      /* PIC_FP64, PIC_MIXED or PIC_COMPENSATED */
  int pusher;         /* PIC_BORIS, PIC_ANALYTIC or PIC_HC */
} pic_batch_desc;

typedef struct {
  int tile[2];              /* field work item in use: x1 strip width, rows per item */
  int grid_blocks;          /* CTAs of the persistent launch */
  int blocks_per_sm;        /* resident CTAs per SM */
  int work_items;           /* field strips + 32-particle chunks (+ corrected rows) per step */
  int graph;                /* 1 if the last run went through a CUDA graph */
  int64_t total_cells;      /* sum over runs of n1*n2 */
  int64_t max_steps;        /* longest run of the last pic_batch_run */
  int64_t cell_steps;       /* sum over runs of n1*n2*nsteps of the last run */
  int64_t particle_steps;   /* sum over runs of particles*nsteps of the last run */
  double last_run_ms;       /* device time of the last pic_batch_run (CUDA events) */
  int has_current;          /* 1 if some particle deposits (two barriers per step) */
  int correction_active;    /* 1 when C^B != e_1 and some particle deposits: each step
                               also applies the x1 current correction (Sec. 3.3) to every
                               row, behind a third barrier */
} pic_batch_info;

/* Create an ensemble; the CFL condition of Eq. (21) is checked for every run's
 * grid (rejecting with PIC_ERR_CFL).  Fields start at zero, no particles.  When
 * C^B != e_1 the x1 current correction of Sec. 3.3 is applied to each run's
 * deposited current as in pic_step, with taps built here for every distinct n1;
 * PIC_ERR_ARG if [k]_B1 vanishes at a grid mode or a row and its taps do not
 * fit in a warp's shared memory (about 12 K FP64 / 24 K FP32 cells). */
pic_status pic_batch_init(const pic_batch_desc* desc, double dt, const pic_coeffs* coeffs,
                          void* stream, pic_batch** out);
/* Per-run laser (nruns entries), loaded as pic_load_laser does. */
pic_status pic_batch_load_laser(pic_batch* b, const pic_laser* lasers);
/* Particles of all runs, grouped by run in run order: counts[r] particles of run
 * r; x = [x1 of all][x2 of all], u = [u1 of all][u2 of all][u3 of all], w
 * (FP64, host).  Positions must lie in each run's box. */
pic_status pic_batch_load_particles(pic_batch* b, const int64_t* counts, const double* x,
                                    const double* u, const double* w, double qm);
/* Steps each run advances per pic_batch_run (nruns entries, >= 0). */
pic_status pic_batch_set_steps(pic_batch* b, const int64_t* nsteps);
/* Time trial_steps of the persistent kernel for each candidate field strip
 * shape and keep the fastest.  Call before loading lasers/particles: it advances the
 * current state and then resets every field to zero. */
pic_status pic_batch_autotune(pic_batch* b, int trial_steps);
/* Set the field strip shape directly (as pic_batch_autotune would): x1 strip
 * width (a positive multiple of 16 bytes of the field type), rows per work
 * item, row stages in each warp's ring (2..8), warps per CTA (1..8).  Results
 * do not depend on it.  PIC_ERR_ARG when out of range or when the rings do not
 * fit in 200 KB of shared memory per CTA (the previous shape is kept). */
pic_status pic_batch_set_strip(pic_batch* b, int width, int rows, int stages, int warps);
/* Advance every run by its step count in one persistent launch (graph replay);
 * synchronises and returns PIC_ERR_TIMEOUT if a grid barrier's bounded wait ran
 * out (the context stays usable). */
pic_status pic_batch_run(pic_batch* b);
/* Read back all particles in the load layout (any pointer may be NULL). */
pic_status pic_batch_read_particles(pic_batch* b, double* x, double* u, double* w);
/* One field component (PIC_E1..PIC_B3 state, or PIC_J*) of run r into an FP64
 * host buffer of n1*n2 values. */
pic_status pic_batch_read_field(pic_batch* b, int run, int comp, double* buf);
/* Fill *info (caller-owned host struct) with the ensemble's shape and the counts
 * and device time of the last pic_batch_run.  PIC_ERR_ARG for null pointers. */
pic_status pic_batch_get_info(pic_batch* b, pic_batch_info* info);
/* Bound of each grid-barrier wait (seconds, default 5).  impossible = 1 makes
 * every barrier wait for one more CTA than the launch has, so that each wait
 * runs out: a test of the timeout path, which must return PIC_ERR_TIMEOUT. */
pic_status pic_batch_set_barrier(pic_batch* b, double timeout_s, int impossible);
/* Message of the ensemble's last failed call ("" if none, or for NULL); the
 * string is owned by the ensemble and valid until its next call. */
const char* pic_batch_last_error(const pic_batch* b);
/* Wait for the ensemble's stream, then free its device memory, graph and the
 * handle itself.  NULL is accepted. */
pic_status pic_batch_destroy(pic_batch* b);

/* Allocation-free laser load.  The paper has no counterpart: this is an
 * interface variant of pic_load_laser for callers that may not allocate device
 * memory themselves -- for example a host application whose GPU memory is owned
 * by another allocator (a framework's caching allocator, or a pool reserved at
 * start-up under a fixed budget), where a library-side cudaMalloc would go
 * around that owner.  It computes the same E2^0 and B3^{-1/2} as
 * pic_load_laser for the given grid, time step and x1 stencil and writes them,
 * in FP64, into the caller's device arrays e2 and b3 (n1*n2*n3 values each,
 * layout as above; the other four components of that state are zero and are
 * not written).  Its only scratch, the two x1 profiles of the pulse, lives in a
 * file-scope device array of 2*PIC_NOALLOC_MAX_N1 doubles (1 MiB), which every
 * GPU that loads the library holds until the process exits; n1 larger than
 * PIC_NOALLOC_MAX_N1 returns PIC_ERR_ARG.  The call makes no cudaMalloc,
 * cudaFree or allocating library call.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current.
 * Every call shares the array
 * and rewrites it in full before reading it; calls that overlap on the GPU
 * (other streams or threads) race on it.  Work runs on `stream` (NULL = legacy
 * default) of the current device; the call returns once the fields are written.
 * Errors: PIC_ERR_ARG (null pointer, bad grid/laser, n1 too large), PIC_ERR_CUDA. */
#define PIC_NOALLOC_MAX_N1 65536
pic_status pic_laser_fields_noalloc(const pic_grid* grid, double dt, const pic_coeffs* coeffs,
                                    const pic_laser* laser, double* e2, double* b3, void* stream);

/* One-line description of the last error of ctx (or of the last failed
 * pic_init when ctx is NULL).  The string is owned by the library. */
const char* pic_last_error(const pic_ctx* ctx);

/* Free the context and its device memory.  NULL is accepted. */
pic_status pic_destroy(pic_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
