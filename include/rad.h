/*
 * rad.h -- C ABI of the B300 (sm_103a) M1 radiation step.
 *
 * One call of rad_step advances the gray M1 radiation field by one explicit
 * transport step followed by the cell-local implicit matter-radiation
 * coupling, as described in Scepi & Lesur, "A nonrelativistic radiative
 * transfer module for Idefix":
 *   - transport: Sect. 2.4 (items 1-7 of the Euler step), Sect. 2.5 (PLM
 *     reconstruction, f-preserving face fix, Eq. f_reconstruct, HLL), Sect. 2.6
 *     (signal speeds lambda_{1,3} and the optically thick correction), Eqs.
 *     (rad1)-(rad2) with the Levermore closure of Sect. 2.1;
 *   - coupling: Sect. 2.8, Eqs. (source_discrete2) and (implicit_matrix),
 *     with the gas energy and momentum from the conservation laws of
 *     Sect. 2.7, Eq. (conservation_energy);
 *   - reduced speed of light c_hat of Sect. 2.7 and the CFL step of Sect. 2.4
 *     item 10.
 * The gas density and velocity are inputs; the step updates the gas internal
 * energy and momentum.
 *
 * Conventions for every function:
 *   - Fields are structure-of-arrays of N = n[0]*n[1]*n[2] cells, x fastest
 *     (cell (i,j,k) at i + n0*(j + n1*k)).  Vector fields (F, v, m) are
 *     `ncomp` consecutive N-arrays in the geometry's orthonormal components:
 *     (x,y,z), (R,phi,z) or (r,theta,phi).
 *   - The element type of every field buffer is double for RAD_FP64 and float
 *     for RAD_FP32_SPLIT (rad_params.precision).
 *   - Pointers marked "host" are read or written only during the call.
 *     Pointers marked "device" must be device memory of the context's device;
 *     the call enqueues work on the context's stream and returns.
 *   - Functions return RAD_OK or an error code and never abort the process.
 *     Device-side failures of an enqueued step (no convergence of the
 *     iteration, non-physical state, bounded waits that ran out) are recorded
 *     in a status word that rad_sync and rad_read return.
 */
#ifndef RAD_H_
#define RAD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RAD_ABI_VERSION 1

typedef enum {
  RAD_OK = 0,
  RAD_EINVAL = 1,       /* invalid argument (pointer, size, value) */
  RAD_ENOMEM = 2,       /* workspace missing or too small, host allocation failed */
  RAD_ECUDA = 3,        /* a CUDA runtime call failed */
  RAD_ENONPHYS = 4,     /* non-physical input or state (E <= 0, |F| > E, NaN) */
  RAD_ENOCONV = 5,      /* the coupling iteration did not converge in some cell */
  RAD_ETIMEOUT = 6,     /* a bounded device wait ran out */
  RAD_EUNSUPPORTED = 7, /* valid request this build does not implement */
  RAD_EBOUNDS = 8       /* debug build only: a device-side index check failed (the
                           access was skipped, the state that step left is not valid) */
} rad_status;

typedef enum { RAD_CARTESIAN = 0, RAD_CYLINDRICAL = 1, RAD_SPHERICAL = 2 } rad_geometry;
/* Boundary conditions (Sect. 3 uses all of them).  The ghost cells of a
 * side are:
 *   OUTFLOW     copies of the edge cell (zero gradient);
 *   PERIODIC    the wrapped cells (both sides of the direction);
 *   REFLECTIVE  mirror images of the cells inside, with the normal flux and
 *               momentum components negated (a wall);
 *   FIXED       a held boundary state (E_b, F_b) and gas temperature T_b
 *               (rad_grid.bc_value), with the edge cell's density: radiation
 *               injection;
 *   LTE         E_r = a_R T_b^4 and gas temperature T_b, F_r copied from
 *               the edge cell (zero gradient), edge-cell density. */
typedef enum {
  RAD_BC_OUTFLOW = 0,
  RAD_BC_PERIODIC = 1,
  RAD_BC_REFLECTIVE = 2,
  RAD_BC_FIXED = 3,
  RAD_BC_LTE = 4
} rad_bc;
typedef enum { RAD_OPAC_CONST = 0, RAD_OPAC_POWERLAW = 1, RAD_OPAC_TABLE = 2 } rad_opac_kind;
/* Precision.  RAD_FP32_SPLIT stores and transports in FP32.  In the
 * coupling it forms the residual E* - a T^4 of the single linearised solve
 * to within one FP32 rounding of its exact value (compensated FP32: T^2 and
 * T^4 carried with their exact FMA remainders, a_R as a pair of floats), as
 * an FP64 evaluation rounded to FP32 would; when iterating (Newton), a T^4,
 * the residual and the numerator of the update are FP64.  The other
 * products of the linearised solve (a T^3, the determinant and its
 * reciprocal, the increments of T and E) are FP32.  It forms f = |F|/E from
 * E^2 and |F|^2 in FP32, so E (and e_floor) must keep E^2 a normal float
 * (E above about 1e-18 in the caller's units); below that use RAD_FP64 or
 * rescale the units. */
typedef enum { RAD_FP64 = 0, RAD_FP32_SPLIT = 1 } rad_precision;
/* Implicit coupling (Sect. 2.8).  RAD_ABSORPTION_ONLY drops the emission by
 * the gas (the first shadow test of Sect. 3): E^{n+1} = E* / (1 + chat dt
 * kappa_P rho), the gas energy following from the conservation of
 * Sect. 2.7; F is updated as in every mode. */
typedef enum { RAD_LINEARIZED_ONCE = 0, RAD_NEWTON = 1, RAD_ABSORPTION_ONLY = 2 } rad_implicit;

/* Face reconstruction (Sect. 2.5): PLM with the van Leer limiter, or LimO3,
 * the compact third-order limited reconstruction, face value
 * u +/- phi(theta) delta / 2 with theta the ratio of the one-sided
 * differences and phi = max(0, min(phi3, max(-theta/2, min(2 theta, phi3,
 * 3/2)))), phi3 = (2 + theta)/3 (index-space differences). */
typedef enum { RAD_PLM = 0, RAD_LIMO3 = 1 } rad_recon;

/* Treatment of reconstructed face states with |F_f| > E_f (Sect. 2.5):
 * FPRESERVE is Eq. (f_reconstruct) (F_f from the cell's F with the cell's
 * f, also applied when f_face <= f_centre); PLUTO takes the cell's flat
 * state (E_c, F_c) where |F_f| > E_f; CLIP rescales F_f to |F_f| = E_f
 * (the plain limiter that Sect. 3's beam test shows to fail). */
typedef enum { RAD_FIX_FPRESERVE = 0, RAD_FIX_PLUTO = 1, RAD_FIX_CLIP = 2 } rad_face_fix;

/* Riemann solver (Sect. 2.5): HLL, or Lax-Friedrichs-Rusanov with the local
 * speed max(|S_L|, |S_R|) of the same thick-limited signal speeds
 * (Sect. 2.6). */
typedef enum { RAD_HLL = 0, RAD_LF = 1 } rad_riemann;

/* Time integration of one step (Sect. 2.4).  RAD_EULER: transport, then
 * the coupling (the step of Sect. 2.4).  RAD_RK2: that split applied in each
 * stage of the two-stage scheme, U1 = S(U^n), U2 = S(U1), U^{n+1} =
 * (U^n + U2) / 2 for the conserved variables E_r, F_r, m and E_gas = e +
 * |m|^2 / (2 rho) (the paper's RK2, which it identifies with IMEX1). */
typedef enum { RAD_EULER = 0, RAD_RK2 = 1 } rad_integrator;

/* Fields for rad_read. */
typedef enum {
  RAD_FIELD_E = 0,    /* radiation energy density E_r, N values */
  RAD_FIELD_F = 1,    /* radiation flux F_r (with the 1/c of Eq. def_flux), ncomp*N */
  RAD_FIELD_EINT = 2, /* gas internal energy density e, N */
  RAD_FIELD_M = 3,    /* gas momentum density rho v, ncomp*N */
  RAD_FIELD_T = 4,    /* gas temperature e / C_v, N */
  RAD_FIELD_RHO = 5   /* gas density, N */
} rad_field;

/* Grid.  Active directions are the first `ndim`; inactive ones have n = 1
 * and their two face coordinates give the extent (e.g. theta in [0, pi]).
 * Angles are in radians.  Face coordinates must increase strictly; radii
 * must be >= 0. */
typedef struct {
  int ndim;                /* 1, 2 or 3 */
  int n[3];                /* cells per direction, >= 1; n[d] = 1 for d >= ndim */
  const double *xface[3];  /* host, n[d]+1 face coordinates each, copied */
  int bc_lo[3], bc_hi[3];  /* rad_bc per active direction; periodic needs both */
  /* boundary state of FIXED and LTE sides: bc_value[d][side] = (E_r, F_0,
   * F_1, F_2, T_b), side 0 lower, 1 upper; FIXED needs E_r > 0, |F| <= E_r
   * and T_b > 0, LTE reads T_b > 0 only; ignored for the other kinds */
  double bc_value[3][2][5];
} rad_grid;

/* Opacity model (per unit mass); the absorption coefficient is kappa*rho.
 * CONST:    kappa_P, kappa_R and sigma as given.
 * POWERLAW: kappa = clip(k0 rho^a_rho T^b_T, kmin, kmax) (Kramers-like,
 *           Sect. 3.3), kappa_P = kappa_R = kappa, sigma = sigma_ratio kappa.
 * TABLE:    log10 kappa on a uniform (log10 rho, log10 T) grid, bilinear in
 *           log space and clamped at the edges; kappa_P = kappa_R = kappa,
 *           sigma = sigma_ratio kappa.  The table is nT rows of nrho values
 *           (rho fastest), host memory, copied. */
typedef struct {
  int kind;
  double kappa_p, kappa_r, sigma;
  double k0, a_rho, b_T, kmin, kmax;
  double sigma_ratio;
  int nrho, nT;
  double lrho0, lrho1, lT0, lT1;
  const float *table_log10_kappa;
} rad_opacity;

/* Physical and numerical parameters (code units, k_B / m_u = 1). */
typedef struct {
  double chat;          /* reduced speed of light, > 0 (Sect. 2.7) */
  double c;             /* speed of light, >= chat */
  double a_rad;         /* radiation constant a_R, > 0 */
  double gamma_gas;     /* adiabatic index, > 1; C_v = rho / (mu (gamma - 1)) */
  double mu;            /* mean molecular weight, > 0 */
  double cfl;           /* Courant number of the fixed CFL step, in (0, 1] */
  double e_floor;       /* floor of E_r, > 0 */
  int precision;        /* rad_precision */
  int implicit_mode;    /* rad_implicit */
  double newton_rtol;   /* RAD_NEWTON: stop when |T_{k+1}-T_k| <= rtol T_{k+1} */
  int newton_maxit;     /* RAD_NEWTON: iteration cap, >= 1 */
  int ncomp;            /* vector components in the caller's F, v and m arrays, 1..3 */
  int use_mlp;          /* RAD_NEWTON only: start the iteration from the learned guess
                           (once rad_mlp_set/init/train has given it parameters) in cells
                           whose first linearised solve changes T by more than mlp_gate */
  double mlp_gate;      /* relative change of T above which the learned guess is used */
  int integrator;       /* rad_integrator */
  int irradiation;      /* 1: the context holds an irradiation deposit field (Sect. 2.9),
                           set with rad_set_irradiation (zero until set) */
  int reconstruction;   /* rad_recon */
  int face_fix;         /* rad_face_fix */
  int riemann;          /* rad_riemann.  Options other than PLM, FPRESERVE and HLL,
                           RAD_ABSORPTION_ONLY and irradiation run on the general
                           form of the step kernel: its register-tiled shapes
                           only (rad_get_launch reports fewer than the default
                           form's on split 3D Cartesian grids) */
  int hydro;            /* 1: evolve the gas too (Cartesian grids; RAD_EUNSUPPORTED
                           otherwise).  Each (sub)step is then a gas step (PLM on
                           rho, v, p; HLL with the Davis speeds; Gamma-law gas),
                           then the radiation transport, then the sources
                           (Sect. 2.4), the radiation reading its optical depths
                           and its gas from the gas step's result.  rad_dt stays
                           the radiation's CFL step: with gas faster than chat
                           the caller passes a smaller dt */
} rad_params;

/* Counters accumulated by rad_step since the last rad_reset_stats. */
typedef struct {
  uint64_t fix;         /* face states whose flux the f-fix recomputed */
  uint64_t efloor;      /* applications of the E floor */
  uint64_t fclip;       /* |F| <= E clips after the coupling */
  uint64_t iters;       /* coupling iterations summed over cells */
  uint64_t itmax;       /* largest iteration count of one cell */
  uint64_t fallback;    /* Newton restarts from T^n */
  uint64_t noconv;      /* cells that did not converge */
  uint64_t steps;       /* steps taken */
} rad_stats;

typedef struct rad_ctx rad_ctx;

/* Fills *p with defaults: chat = c = 1, a_rad = 1, gamma = 5/3, mu = 1,
 * cfl = 0.4, e_floor = 1e-30, RAD_FP64, RAD_LINEARIZED_ONCE, rtol = 1e-12,
 * maxit = 50, ncomp = 3, use_mlp = 0, mlp_gate = 1e-2, RAD_EULER, irradiation = 0,
 * RAD_PLM, RAD_FIX_FPRESERVE, RAD_HLL, hydro = 0.  Returns RAD_EINVAL if
 * p is NULL. */
rad_status rad_default_params(rad_params *p);

/* Validates the description, precomputes the geometry (face areas, volumes,
 * metric factors, the CFL step of Sect. 2.4 item 10) on the host and
 * returns a context that owns no device memory yet.  Host arrays are copied.
 * Errors: RAD_EINVAL for any invalid field, RAD_ENOMEM if host allocation
 * fails.  *out is set only on success. */
rad_status rad_create(const rad_grid *grid, int geometry, const rad_opacity *opacity,
                      const rad_params *params, rad_ctx **out);

/* Device bytes the context needs (double-buffered state with ghost layers,
 * geometry tables, opacity table, counters, staging for host copies). */
rad_status rad_workspace_size(const rad_ctx *ctx, size_t *bytes);

/* Binds caller-owned device memory of at least rad_workspace_size bytes,
 * 256-byte aligned, on the current device; the caller keeps it alive until
 * rad_destroy.  Errors: RAD_EINVAL (NULL, misaligned), RAD_ENOMEM (too
 * small), RAD_ECUDA. */
rad_status rad_bind_workspace(rad_ctx *ctx, void *device_ptr, size_t bytes);

/* Convenience for C callers: allocates the workspace with cudaMalloc (freed
 * by rad_destroy).  Errors: RAD_ENOMEM, RAD_ECUDA. */
rad_status rad_alloc_workspace(rad_ctx *ctx);

/* Sets the CUDA stream (a cudaStream_t) on which all work is enqueued;
 * NULL selects the legacy default stream. */
rad_status rad_set_stream(rad_ctx *ctx, void *cuda_stream);

/* Sets the gas: rho (N), v (ncomp*N) and T (N), all host (on_device = 0)
 * or all device (on_device = 1).  Stores rho, m = rho v and e = C_v T.
 * The call returns after the copies completed.  Errors: RAD_EINVAL (NULL, no
 * workspace), RAD_ENONPHYS (a value that is not finite, or rho or T not
 * positive; the state is stored as given and should be replaced),
 * RAD_ECUDA. */
rad_status rad_set_gas(rad_ctx *ctx, const void *rho, const void *v, const void *T,
                       int on_device);

/* Sets the radiation field: E (N) and F (ncomp*N), host or device, and
 * returns after the copies completed.  Errors as rad_set_gas: RAD_ENONPHYS
 * for a value that is not finite or an E that is not positive (|F| > E is
 * accepted: the closure clamps f at 1). */
rad_status rad_set_rad(rad_ctx *ctx, const void *E, const void *F, int on_device);

/* Enqueues nsteps steps of size dt (dt <= 0: the CFL step of rad_dt).
 * Asynchronous on the context's stream.  Errors: RAD_EINVAL (nsteps < 0, no
 * state set), RAD_ECUDA (launch failure). */
rad_status rad_step(rad_ctx *ctx, double dt, int nsteps);

/* Copies a field (rad_field) into dst of `bytes` bytes (host or device).
 * Synchronises the stream for host destinations and returns the device
 * status word (RAD_ENOCONV, RAD_ENONPHYS, ...) if a step recorded one.
 * Errors: RAD_EINVAL (unknown field, bytes too small). */
rad_status rad_read(rad_ctx *ctx, int field, void *dst, size_t bytes, int on_device);

/* Asynchronous host transfers, for callers that stream a state through the
 * GPU every step (the paper has no counterpart; it is a transfer pattern of
 * this library).  They take host pointers only, best in pinned memory, and
 * return as soon as the work is enqueued: the host buffers must stay valid
 * and must not be read (outputs) or changed (inputs) until rad_sync
 * returns.  Uploads run on an upload stream of the context, read-backs on a
 * read-back stream, ordered with the steps on the context's stream by
 * events, so that the read-back of one step overlaps the upload of the
 * next.  Each call uses a staging area of its own: the first call
 * allocates it (cudaMalloc of (7 + 4 ncomp) N values) together with the
 * two streams, and rad_destroy frees them.
 *   rad_set_gas_host_async: as rad_set_gas with host rho (N), v (ncomp*N),
 *   T (N).
 *   rad_set_rad_host_async: as rad_set_rad with host E (N), F (ncomp*N).
 *   rad_read_host_async: as rad_read into host dst; the value is the state
 *   after the steps enqueued before the call.
 * Errors: RAD_EINVAL (NULL, unknown field, bytes too small, no state set
 * before a read), RAD_ENOMEM (no workspace, or the staging allocation
 * failed), RAD_ECUDA.  Device status words, and RAD_ENONPHYS for
 * non-physical uploaded values (as rad_set_gas / rad_set_rad), surface at
 * rad_sync. */
rad_status rad_set_gas_host_async(rad_ctx *ctx, const void *rho, const void *v, const void *T);
rad_status rad_set_rad_host_async(rad_ctx *ctx, const void *E, const void *F);
rad_status rad_read_host_async(rad_ctx *ctx, int field, void *dst, size_t bytes);

/* Irradiation by an external source (Sect. 2.9): q = -div F_irr, the energy
 * the irradiation flux deposits per unit volume and time, N values (flat, x
 * fastest, the precision of the context), host or device.  Each step adds
 * dt q to the gas row of the implicit solve and to the gas energy, so that
 * E_gas + (c/chat) E_r gains dt q.  The field stays until set again.
 * Requires params.irradiation = 1 at rad_create.  Errors: RAD_EINVAL (no
 * irradiation field, NULL q), RAD_ENOMEM, RAD_ENONPHYS (a value that is
 * not finite), RAD_ECUDA. */
rad_status rad_set_irradiation(rad_ctx *ctx, const void *q, int on_device);

/* Waits for the stream and returns the device status word (RAD_OK if no
 * step recorded a failure); the word is cleared by the read. */
rad_status rad_sync(rad_ctx *ctx);

/* The CFL step dt = cfl / max_cells sum_d (chat / h_d), h_d the physical
 * cell widths. */
rad_status rad_dt(const rad_ctx *ctx, double *dt);

/* Reads (synchronising) and resets the counters. */
rad_status rad_get_stats(rad_ctx *ctx, rad_stats *out);
rad_status rad_reset_stats(rad_ctx *ctx);

/* Number of kernel launches rad_step enqueues per step (for launch
 * accounting by callers). */
int rad_launches_per_step(const rad_ctx *ctx);

/* Kernel timing (not in the paper: a measurement aid).  After
 * rad_profile_begin, each of the next max_steps steps records CUDA events on
 * the stream around its step kernel and around its queue pass (RAD_NEWTON).
 * rad_profile_end waits for the last of them and returns the summed device
 * times (ms) of the step kernels and of the queue passes and the number of
 * steps timed (any output may be NULL), then releases the events.  Errors:
 * RAD_EINVAL (max_steps outside 1..2^20), RAD_ECUDA. */
rad_status rad_profile_begin(rad_ctx *ctx, int max_steps);
rad_status rad_profile_end(rad_ctx *ctx, float *step_ms, float *queue_ms, int *nsteps);

/* Launch shape of the step kernel: `variant` selects one of the CTA shapes
 * instantiated for this grid (0 = default; rad_get_launch reports how many)
 * and `chunk` the number of cells a CTA marches along the slowest active
 * axis (0 = default).  Results do not depend on either.  Not in the paper:
 * a tuning knob of this implementation.  Errors: RAD_EINVAL. */
rad_status rad_set_launch(rad_ctx *ctx, int variant, int chunk);
rad_status rad_get_launch(const rad_ctx *ctx, int *variant, int *chunk, int *nvariants);

/* Bound on the first wait of the TMA-staged step kernels for each plane of
 * the state (the launch variants that stage planes by TMA; the others do not
 * wait).  0 (the default) is a bounded blocking wait of 2^21 tries, far
 * longer than a copy takes; polls > 0 makes it that many non-blocking tests
 * of the plane's mbarrier.  A wait that runs out stops the CTA once its
 * copies in flight have landed, and the next rad_sync returns RAD_ETIMEOUT.
 * The state that step leaves is not valid (set it again), but the context
 * stays usable.  Not in the paper: it exists so that the timeout path can be
 * exercised without a fault.  Errors: RAD_EINVAL. */
rad_status rad_set_wait_limit(rad_ctx *ctx, unsigned int polls);

/* Debug build (librad_debug.so, built with RAD_DEBUG_CHECKS): every store
 * of the step kernels and the gas step checks its cell index against the
 * padded arrays; a failed check sets a flag that the next rad_sync returns
 * as RAD_EBOUNDS, and the access is skipped (no trap).  Not in the paper: it
 * stands in for a memory checker.  rad_debug_check_index runs one such
 * check on the context's stream, on E of the current state at cell `index`
 * of the padded layout (rewriting the value it holds when the index is in
 * range), so that the check itself can be exercised; release builds do
 * nothing and return RAD_EUNSUPPORTED.  Errors: RAD_EINVAL, RAD_ENOMEM,
 * RAD_ECUDA. */
rad_status rad_debug_check_index(rad_ctx *ctx, long long index);

/* Autotuner: times `reps` steps of every (shape, chunk) candidate on the
 * current state without advancing it (each trial recomputes the same step
 * into the spare buffer), selects the fastest, and restores the counters
 * and the status word.  Outputs (any may be NULL): the chosen variant and
 * chunk and its time per step in ms.  Synchronises the stream.  Not in the
 * paper.  Errors: RAD_EINVAL (no state), RAD_ENOMEM, RAD_ECUDA. */
rad_status rad_tune(rad_ctx *ctx, int reps, int *variant, int *chunk, float *ms);

/* --------------------------------------------------------------------------
 * Learned starting guess of the coupling iteration (not in the paper: an
 * extension of this implementation).  In RAD_NEWTON mode the root T^{n+1}
 * of the cell's coupling depends only on alpha = g a T^n^3/((1+g_r) C_v) and
 * eps = E* / (a T^n^4) (Sect. 2.8 with T^4 kept exact).  A network with three
 * tanh layers of 64 units maps (log10 alpha / 4, log10 eps / 4) to
 * log(T^{n+1}/T^n); the iteration starts from T^n exp(output) and keeps its
 * convergence test, so results agree with starting from T^n to that test.
 * Records are float4 (x1, x2, log(T^{n+1}/T^n), gate value), device memory,
 * and every record pointer must be 16-byte aligned (an offset view of a
 * record array that starts inside a record is refused with RAD_EINVAL).
 * Parameters: rad_mlp_nparam() floats, laid out W1 (64x2, row-major), b1,
 * W2 (64x64), b2, W3 (64x64), b3, w4 (64), b4.
 * -------------------------------------------------------------------------- */
int rad_mlp_nparam(void);

/* Host copies of the parameters in and out (n == rad_mlp_nparam()); set
 * also clears the Adam moments.  Errors: RAD_EINVAL, RAD_ENOMEM, RAD_ECUDA. */
rad_status rad_mlp_set(rad_ctx *ctx, const float *host_params, size_t n);
rad_status rad_mlp_get(rad_ctx *ctx, float *host_params, size_t n);

/* Glorot-uniform weights, zero biases, from a seeded splitmix64 stream. */
rad_status rad_mlp_init(rad_ctx *ctx, uint64_t seed);

/* Trains on n device records: `epochs` passes over a seeded permutation of
 * the records in mini-batches of `batch`, mean-squared error, Adam with step
 * lr.  Runs forward/backward/update kernels on the context's stream and
 * synchronises; *final_loss (may be NULL) is the mean loss of the last epoch.
 * Initialises the parameters first if none were given. */
rad_status rad_mlp_train(rad_ctx *ctx, const float *dev_records, size_t n, int epochs, int batch,
                         float lr, uint64_t seed, float *final_loss);

/* Gradient of the mean-squared error over n device records with the current
 * parameters (host_grad: rad_mlp_nparam() floats, may be NULL) and the loss;
 * synchronises.  For checking the training kernels. */
rad_status rad_mlp_grad(rad_ctx *ctx, const float *dev_records, size_t n, float *host_grad,
                        float *host_loss);

/* Network output for n device records into dev_out (n floats).
 * rad_mlp_predict evaluates in FP32 on the CUDA cores; rad_mlp_predict_tc
 * evaluates as the queue pass does, with the two hidden 64 x 64 layers on the
 * tensor cores (bf16 operands, FP32 accumulation: about three significant
 * digits).  A bounded wait of the tensor-core path that ran out is reported
 * as RAD_ETIMEOUT by the next rad_sync. */
rad_status rad_mlp_predict(rad_ctx *ctx, const float *dev_records, size_t n, float *dev_out);
rad_status rad_mlp_predict_tc(rad_ctx *ctx, const float *dev_records, size_t n, float *dev_out);

/* Logging of converged RAD_NEWTON solves for training: cells whose linear
 * index is a multiple of `stride` append one record to dev_records (up to
 * `capacity`); NULL unbinds.  rad_log_count returns the records written
 * (synchronising). */
rad_status rad_log_bind(rad_ctx *ctx, float *dev_records, size_t capacity, long long stride);
rad_status rad_log_count(rad_ctx *ctx, size_t *n);

/* --------------------------------------------------------------------------
 * Gradient of the learned guess's training loss without device allocation.
 * The paper has no counterpart: this is a convenience of this library.
 *
 * Same result as rad_mlp_grad (mean-squared-error gradient and mean loss over
 * n records, for the parameters at dev_params), but it takes no context and
 * allocates nothing.  It is meant for callers that cannot allocate device
 * memory when they need the gradient: code whose framework owns all device
 * memory through a pre-sized pool and forbids allocations after start-up, or
 * code that must not let cudaMalloc/cudaFree synchronise the device.
 *
 * dev_params: rad_mlp_nparam() floats; dev_records: n float4 records (x1,
 * x2, target, unused); dev_grad: rad_mlp_nparam() floats and dev_loss: one
 * float, all device memory of the current device; the work is enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default stream) and the call
 * returns without waiting.
 *
 * Scratch: a file-scope device array of RAD_NOALLOC_MAX_RECORDS /
 * RAD_NOALLOC_ROW_RECORDS partial gradients (about 8.8 MB) that every GPU
 * loading this library holds until the process exits.  Each call sums one
 * partial per RAD_NOALLOC_ROW_RECORDS records in a fixed order, so the result
 * is deterministic; every partial a call uses is fully rewritten, so nothing
 * left by an earlier call leaks into it.  All calls share the array: calls
 * that overlap on the GPU (other streams, other threads) race and give wrong
 * results; order them on one stream.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.
 *
 * Errors: RAD_EINVAL for NULL pointers, dev_records not 16-byte aligned,
 * n == 0 or n > RAD_NOALLOC_MAX_RECORDS
 * (split larger sets and add the gradients, weighted by their counts);
 * RAD_EUNSUPPORTED for device ordinals >= 64; RAD_ECUDA if the address lookup
 * or a launch fails. */
#define RAD_NOALLOC_ROW_RECORDS 64
#define RAD_NOALLOC_MAX_RECORDS 16384
rad_status rad_mlp_grad_noalloc(const float *dev_params, const float *dev_records, size_t n,
                                float *dev_grad, float *dev_loss, void *stream);

/* --------------------------------------------------------------------------
 * Batches: many independent grids advanced together (not in the paper: an
 * extension of this implementation for serving many small problems).  Each
 * step of every grid is one launch of a persistent kernel whose CTAs take
 * tiles of any grid from a shared work list (largest grids first), so small
 * grids do not leave the GPU idle; in RAD_NEWTON mode a second launch runs
 * the queue pass over all grids.  A sequence of steps is captured once into a
 * CUDA graph and replayed.  Each grid gets the values it gets from rad_step.
 *
 * Members are contexts made by rad_create with a bound workspace and their
 * gas and radiation set; all are Cartesian with the same ndim (2 or 3),
 * precision, ncomp, implicit mode and use_mlp, use RAD_EULER, and all have
 * constant widths
 * along each direction or all do not.  The batch does not own them: they
 * must outlive it, and rad_set_gas / rad_set_rad / rad_read on a member
 * stay valid between batch steps (rad_batch_set_stream puts every member on
 * the batch's stream).  Batch steps add to the batch's counters, not to the
 * members'.
 * -------------------------------------------------------------------------- */
typedef struct rad_batch rad_batch;

/* Validates the members (1..1024 distinct contexts) and returns a batch that
 * owns no device memory yet.  Errors: RAD_EINVAL, RAD_EUNSUPPORTED (members
 * that differ in kind, or a kind without batched kernels: non-Cartesian,
 * RAD_RK2, face options other than the defaults, RAD_ABSORPTION_ONLY,
 * irradiation), RAD_ENOMEM. */
rad_status rad_batch_create(rad_ctx *const *members, int count, rad_batch **out);

/* Device memory the batch needs for its own state: the members' argument
 * blocks, the tile work list, counters, queue lengths and the network
 * parameters (the members keep their own workspaces).  Binding follows the
 * rules of rad_bind_workspace (256-byte aligned, caller-owned). */
rad_status rad_batch_workspace_size(const rad_batch *b, size_t *bytes);
rad_status rad_batch_bind_workspace(rad_batch *b, void *dev_ptr, size_t bytes);
rad_status rad_batch_alloc_workspace(rad_batch *b);

/* Stream of the batch and of every member (NULL = legacy default stream). */
rad_status rad_batch_set_stream(rad_batch *b, void *stream);

/* use_graph != 0 (default): rad_batch_step captures its sequence of launches
 * into a CUDA graph on a private stream the first time a given step count is
 * asked for, and replays it on the batch's stream; 0: plain launches. */
rad_status rad_batch_set_graph(rad_batch *b, int use_graph);

/* Enqueues nsteps steps of every member.  dt: host array of one step length
 * per member (entries <= 0, or dt == NULL, use the member's CFL step).
 * Asynchronous; device failures land in the batch status word.  Errors:
 * RAD_EINVAL (member without state, bad dt), RAD_ENOMEM, RAD_ECUDA. */
rad_status rad_batch_step(rad_batch *b, const double *dt, int nsteps);

/* Waits for the stream and returns (and clears) the batch status word. */
rad_status rad_batch_sync(rad_batch *b);

/* Counters summed over all members for the batch steps; steps counts batch
 * steps.  Reading synchronises. */
rad_status rad_batch_get_stats(rad_batch *b, rad_stats *out);
rad_status rad_batch_reset_stats(rad_batch *b);

/* Kernel launches per batch step (1, or 2 in RAD_NEWTON mode). */
int rad_batch_launches_per_step(const rad_batch *b);

/* CTA shape (`variant`, see rad_batch_get_launch for the count) and march
 * length (`chunk`, 0 = default) of the persistent kernel; results do not
 * depend on either.  rad_batch_get_launch also reports the CTAs of the last
 * launch configuration (0 before the first step).  Errors: RAD_EINVAL. */
rad_status rad_batch_set_launch(rad_batch *b, int variant, int chunk);
rad_status rad_batch_get_launch(const rad_batch *b, int *variant, int *chunk, int *nvariants,
                                int *blocks);

/* Autotuner of the persistent launch: times `reps` launches of every
 * (shape, chunk) pair on the current state without advancing it, keeps the
 * fastest and restores the counters and the status word; synchronises.
 * Outputs may be NULL. */
rad_status rad_batch_tune(rad_batch *b, int reps, int *variant, int *chunk, float *ms);

/* Parameters of the learned guess used by every member (use_mlp members;
 * layout as for rad_mlp_set).  Errors: RAD_EINVAL (wrong n, members without
 * use_mlp), RAD_ENOMEM, RAD_ECUDA. */
rad_status rad_batch_mlp_set(rad_batch *b, const float *host_params, size_t n);

/* Releases the batch (not the members). */
void rad_batch_destroy(rad_batch *b);

/* Releases the context (and the workspace if rad_alloc_workspace made it). */
void rad_destroy(rad_ctx *ctx);

/* Static description of a status code. */
const char *rad_strerror(rad_status s);

#ifdef __cplusplus
}
#endif
#endif /* RAD_H_ */
