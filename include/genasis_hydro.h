/*
 * genasis_hydro.h -- C ABI of the GB300 (sm_103a) finite-volume update of
 * nonrelativistic ideal hydrodynamics described in Cardall, Budiardja, Endeve
 * & Mezzacappa, "GenASiS: General Astrophysical Simulation System. I.
 * Refinable mesh and nonrelativistic hydrodynamics" (arXiv:1207.3392).
 *
 * The library advances the balance equations dU/dt = L[U] (Eq. BalanceEquation,
 * no sources) on one single-level Cartesian mesh with non-uniform widths per
 * axis:
 *   - primitive recovery n = D, v = S / (m D), e = G - m n |v|^2 / 2,
 *     p = (gamma - 1) e, m = 1                           (Sec. 3.5)
 *   - limited linear reconstruction, Eq. MinMod with parameter theta  (Sec. 3.1)
 *   - HLL (Eq. FluxHLL) or HLLC (Eqs. MiddleWaveSpeed..FluxHLLC) face fluxes (Sec. 3.2, 3.5)
 *   - flux divergence, Eq. BalanceEquationAverage with A_q / V = 1 / dq
 *   - second-order TVD Runge-Kutta (Heun), Eqs. Update, RungeKutta1-3  (Sec. 3.4)
 *   - CFL time step, Eq. courantTimeStep times C_CFL      (Sec. 3.6)
 *
 * Conventions for every entry point
 *   - Arrays are structure-of-arrays, C order, x fastest: element (v, k, j, i)
 *     of a field with nv components sits at ((v * nz + k) * ny + j) * nx + i,
 *     with ny = nz = 1 below 3D (nz = 1 in 2D).  Conserved fields have
 *     nv = ndim + 2 components (D, S_1..S_ndim, G).
 *   - Pointers marked "host or device" may point to host memory (pageable or
 *     pinned) or to device memory of the current device; the library detects
 *     which.  The caller keeps ownership of every pointer it passes; the
 *     library copies what it needs before the call returns (or, for device
 *     pointers, in stream order before the next call's work).
 *   - The library owns all device state of a handle and frees it in
 *     genasis_hydro_destroy.
 *   - All work runs on the handle's CUDA stream.  Calls that return numbers to
 *     the host (compute_dt, get_*, status) synchronise that stream; the others
 *     are asynchronous.
 *   - Every call returns GENASIS_OK or a negative error code and never aborts.
 *     genasis_hydro_last_error() describes the last failure of the calling
 *     thread.  A non-physical state (rho <= 0, p <= 0, or a non-finite value)
 *     detected on the device sets a sticky status reported by
 *     genasis_hydro_status and by every later synchronising call.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef GENASIS_HYDRO_H
#define GENASIS_HYDRO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GENASIS_OK 0
#define GENASIS_EINVAL (-1)    /* bad argument */
#define GENASIS_ENOMEM (-2)    /* device allocation failed */
#define GENASIS_ECUDA (-3)     /* CUDA runtime error */
#define GENASIS_ENONPHYS (-4)  /* rho <= 0, p <= 0 or non-finite value met on the device */
#define GENASIS_ETIMEOUT (-5)  /* a bounded device wait gave up */

#define GENASIS_HLL 0
#define GENASIS_HLLC 1
/* HLLC, switching to HLL in the vicinity of a shock on the faces transverse to
 * its motion (Sec. 3.2; the detector, which the paper does not give, is: a
 * cell lies on a shock moving along axis r when, across its two neighbours
 * along r, v_r decreases and the pressure jumps by more than half the smaller
 * pressure; a face normal to q takes HLL when either of its cells lies on a
 * shock moving along an axis other than q).  The bits come from each RK
 * stage's input state.  2D and 3D, GENASIS_FP64 or GENASIS_FP32_MIXED; in 1D
 * it is plain HLLC. */
#define GENASIS_HLLC_SWITCH 2

#define GENASIS_BC_PERIODIC 0  /* wrap-around */
#define GENASIS_BC_REFLECT 1   /* mirror, normal momentum negated */
#define GENASIS_BC_OUTFLOW 2   /* copy of the edge cell */

#define GENASIS_FP64 0         /* state stored and processed in FP64 */
#define GENASIS_FP32_MIXED 1   /* state stored and fluxes in FP32 (FP32 results
                                  below 2^-126 flush to zero); internal-energy
                                  cancellation, dt and totals reductions in FP64 */
#define GENASIS_FP64_DW 2      /* state and arithmetic as double-word pairs of FP32
                                  (hi + lo, ~48 bits) on the FP32 pipes; the same
                                  results as GENASIS_FP64 to ~1e-13; host arrays are
                                  FP64 (or FP32) and converted on the device */

typedef struct genasis_hydro *genasis_hydro_t;

/* Mesh and solver description (Sec. 2 mesh, single level; Secs. 3.1-3.5).
 *   ndim        1, 2 or 3
 *   n[q]        cells along axis q (>= 2 on active axes; ignored beyond ndim)
 *   widths[q]   host pointer to n[q] strictly positive cell widths along q
 *   origin[q]   coordinate of the low face of cell 0 along q; the update does
 *               not depend on it (Eq. BalanceEquationAverage needs only the
 *               widths); genasis_hydro_get_centers returns the cell centres
 *               measured from it
 *   bc_lo/hi[q] GENASIS_BC_* at the low / high end of axis q (periodic must be
 *               set on both ends)
 *   gamma       adiabatic index of p = (gamma - 1) e (> 1)
 *   solver      GENASIS_HLL or GENASIS_HLLC
 *   theta       slope limiter parameter of Eq. MinMod, in [1, 2] (paper: 1.4)
 *   precision   GENASIS_FP64, GENASIS_FP32_MIXED or GENASIS_FP64_DW
 *   stream      cudaStream_t to run on, or NULL for a stream owned by the handle */
typedef struct {
  int ndim;
  int n[3];
  const double *widths[3];
  double origin[3];
  int bc_lo[3];
  int bc_hi[3];
  double gamma;
  int solver;
  double theta;
  int precision;
  void *stream;
} genasis_hydro_desc;

/* Create a handle: validates desc, allocates the device state (two state
 * buffers, the stage buffer, geometry tables, reduction partials) and picks
 * the default tile shape.  The state is zero until set_primitive or
 * set_conserved.  Returns EINVAL on a bad description, ENOMEM, ECUDA. */
int genasis_hydro_create(const genasis_hydro_desc *desc, genasis_hydro_t *out);

/* Release every device resource of h (synchronises its stream).  NULL is OK. */
int genasis_hydro_destroy(genasis_hydro_t h);

/* Set the state from primitives (Eqs. BalancedBaryonDensity, MomentumDensity,
 * balancedEnergy with p = (gamma-1) e): rho[ncell], vel[ndim * ncell] (one
 * plane per axis), p[ncell]; FP64, host or device.  Resets time to 0.
 * Device inputs are read on the handle's stream: work on other streams that
 * writes them must be complete (or ordered before it) when this is called;
 * the same holds for every call below that takes device pointers. */
int genasis_hydro_set_primitive(genasis_hydro_t h, const double *rho, const double *vel, const double *p);

/* Set / read the conserved state U[(ndim + 2) * ncell] in the given precision
 * (GENASIS_FP64 = double, GENASIS_FP32_MIXED = float), host or device,
 * converting if it differs from the handle's.  get_conserved synchronises. */
int genasis_hydro_set_conserved(genasis_hydro_t h, const void *U, int precision);
int genasis_hydro_get_conserved(genasis_hydro_t h, void *U, int precision);

/* The same copies, enqueued on the handle's stream without synchronising, so
 * that transfers of one handle overlap the steps of another (the paper has no
 * counterpart; it is the host <-> device side of the boundary).  A host U
 * should be page-locked (otherwise the copy is staged and may not overlap);
 * it must stay valid and unchanged until genasis_hydro_sync(h) returns.  The
 * non-physical status is reported by genasis_hydro_sync, not here. */
int genasis_hydro_set_conserved_async(genasis_hydro_t h, const void *U, int precision);
int genasis_hydro_get_conserved_async(genasis_hydro_t h, void *U, int precision);
/* Wait for all work enqueued on h's stream; returns ENONPHYS / ETIMEOUT if the
 * sticky status is set, else OK. */
int genasis_hydro_sync(genasis_hydro_t h);

/* dt = cfl * dt_CFL of the current state (Eq. courantTimeStep); synchronises. */
int genasis_hydro_compute_dt(genasis_hydro_t h, double cfl, double *dt);

/* One full RK2 step (Eqs. RungeKutta1-3) with the given dt (> 0); asynchronous. */
int genasis_hydro_step(genasis_hydro_t h, double dt);

/* nsteps RK2 steps, each with dt = cfl * dt_CFL taken on the device from the
 * state at the start of the step; if t_end > 0 the last step is shortened so
 * that time stops exactly at t_end and later steps do nothing (Algorithm
 * Evolve, single level).  Runs as one CUDA graph launch (captured on first use
 * per (nsteps, cfl, t_end)).  If t_out is non-NULL it synchronises and stores
 * the time reached. */
int genasis_hydro_advance(genasis_hydro_t h, int nsteps, double cfl, double t_end, double *t_out);

/* Current time (synchronises) / reset the time counter. */
int genasis_hydro_get_time(genasis_hydro_t h, double *t);
int genasis_hydro_set_time(genasis_hydro_t h, double t);

/* Volume-integrated conserved totals sum_cells U dV, FP64, of the current
 * state: totals[0 .. ndim + 1] (Sec. 3.3 conservation tally).  Synchronises. */
int genasis_hydro_get_totals(genasis_hydro_t h, double *totals);

/* Synchronise and return GENASIS_ENONPHYS if the sticky device status is set,
 * else GENASIS_OK; clear_status resets it. */
int genasis_hydro_status(genasis_hydro_t h);
int genasis_hydro_clear_status(genasis_hydro_t h);

/* Launch configuration: tile index (0 .. tile_count - 1 for this ndim) and
 * planes per CTA along the march axis (0 = automatic).  info[0..5] receives
 * (tile index, tile x, tile y, planes per CTA, CTAs per stage, tile count).
 * Tile x and y count the cells a CTA owns: in 1D/2D a CTA of n threads owns
 * n - 1 columns (its last thread loads the next tile's first cell as a
 * neighbour only). */
int genasis_hydro_set_tile(genasis_hydro_t h, int tile, int kchunk);
int genasis_hydro_get_tile(genasis_hydro_t h, int *info);

/* Time every compiled tile shape (and a few plane counts) on the current
 * state for `trial_steps` steps each, keep the fastest, restore the state.
 * It chooses among the tiles that give bitwise the same states as the
 * default tile; the 3D FP32 tiles that take two march planes per thread on
 * the packed FP32 instructions (tiles 11 to 13: the same arithmetic with
 * other roundings) are chosen only with genasis_hydro_set_tile.
 * If cache_path is non-NULL the choice is read from / appended to that text
 * file, keyed by (ndim, n, precision, solver).  Synchronises. */
int genasis_hydro_autotune(genasis_hydro_t h, int trial_steps, const char *cache_path);

/* Handle options.  GENASIS_OPT_STEP_TOTALS: 1 (default) folds the FP64
 * conserved totals of U^n into stage 1 of every step (readable after the step
 * with genasis_hydro_get_step_totals); 0 skips that work.  Returns EINVAL for
 * an unknown option or value. */
#define GENASIS_OPT_STEP_TOTALS 1
/* GENASIS_OPT_ONE_LAUNCH: 1 (default) runs genasis_hydro_step and
 * genasis_hydro_advance of a 1D FP64 or FP32-mixed HLL/HLLC mesh of at most
 * 4088 cells as one cooperative kernel launch (one CTA per tile, bounded grid
 * barriers between the phases) for all the steps of the call
 * (the same tile arithmetic and dt fold as the three launches per step, so
 * bitwise the same states, dt and time; the step totals sum the cells in
 * tiles of another width and agree to rounding); 0 keeps three launches per
 * step.  With a network attached (genasis_hydro_set_flux_mlp) the option is
 * passed on to its corrected scheme (genasis_learned_set_option), as is
 * GENASIS_OPT_MLP_TCGEN05 (defined with genasis_learned_set_option), which
 * this call also accepts. */
#define GENASIS_OPT_ONE_LAUNCH 2
int genasis_hydro_set_option(genasis_hydro_t h, int option, int value);
/* External force of a linear potential Phi = grad_phi . x (the uniform force
 * of the Rayleigh-Taylor test, Sec. 4.3.2): each stage adds the source
 * S_q = -D dPhi/dq to the momenta and -sum_q S_q dPhi/dq to the energy,
 * from each cell's stage-input state (the paper prints the source vector
 * without its sign; the force is -grad Phi).  grad_phi[3] (entries beyond
 * ndim are ignored); all zero turns the source off (the default).  Returns
 * EINVAL for a non-finite entry. */
int genasis_hydro_set_potential_gradient(genasis_hydro_t h, const double *grad_phi);
/* Totals of U^n of the last step taken with GENASIS_OPT_STEP_TOTALS = 1
 * (totals[0 .. ndim + 1]); synchronises. */
int genasis_hydro_get_step_totals(genasis_hydro_t h, double *totals);

/* Number of kernel launches one step enqueues. */
int genasis_hydro_launches_per_step(genasis_hydro_t h);

/* One CFL step like genasis_hydro_advance(h, 1, cfl, 0, NULL), launched
 * kernel by kernel with CUDA events around each launch on the handle's stream;
 * ms[0..2] receive the device durations of stage 1, the dt/totals
 * finalisation and stage 2 (milliseconds).  Synchronises. */
int genasis_hydro_profile_step(genasis_hydro_t h, double cfl, float *ms);

/* Text of the last error of the calling thread (never NULL). */
const char *genasis_hydro_last_error(void);

/* Geometric cell centres along axis q (0 .. ndim - 1) of a single-mesh
 * handle: x[i] = origin[q] + sum_{j < i} widths[q][j] + widths[q][i] / 2
 * (Sec. 3.1: the reconstruction is about the geometric centre), n[q] doubles
 * into host memory. */
int genasis_hydro_get_centers(genasis_hydro_t h, int axis, double *x);

/* Vector FMA throughput of the current GPU in TFLOP/s (2 operations per
 * FMA), measured with independent FMA chains on every SM under CUDA events:
 * kind 0 FP64, 1 FP32, 2 FP32 with the packed two-lane FMA of sm_100+.  The
 * paper has no counterpart: it is the measured denominator of the arithmetic
 * roofline that the update's kernels are reported against.  Allocates and
 * frees a small buffer, uses a private stream, takes ~0.5 s; synchronises. */
int genasis_measure_fma_rate(int kind, double *tflops);
/* Host-link copy rate in GB/s (the paper has no counterpart: the measured
 * denominator of the end-to-end roofline, whose steps copy the state in and
 * out): 256 MiB page-locked host buffers copied with cudaMemcpyAsync, kind 0
 * host to device, 1 device to host, 2 both directions at once on two
 * streams (the rate of the two together).  Allocates and frees ~1 GB (half
 * page-locked host memory), uses private streams, takes ~0.1 s; synchronises. */
int genasis_measure_link_rate(int kind, double *gbs);

/* Check that the kernels' bounded waits give up instead of hanging (the paper
 * has no counterpart: a diagnostic of this library).  Runs two waits that
 * cannot complete, on the legacy default stream: a grid barrier of two CTAs of
 * which only one arrives (the barrier of the one-launch advances), and an
 * mbarrier that nothing arrives on (the wait of the TMA and tcgen05 kernels).
 * status[0], status[1] receive their status words: 2 (the timeout bit) when
 * the wait gave up, 0 if it (impossibly) completed; seconds[0], seconds[1]
 * their event-timed durations, about one second each.  No fault or trap is
 * involved and the context stays usable.  Synchronises; ~2 s. */
int genasis_check_bounded_waits(unsigned *status, double *seconds);

/* ---------------------------------------------------------------------------
 * The batched and learned workloads behind genasis_hydro_t.
 *
 * genasis_hydro_batch_create makes one handle for nprob independent 1D or 2D
 * problems, each described by its own genasis_hydro_desc (ndim 1 or 2, n,
 * widths, boundaries, gamma); solver, theta, precision and stream must be the
 * same in every desc (EINVAL otherwise).  Each problem follows the update of
 * a single-mesh handle (Secs. 3.1-3.6) with its own CFL time step; the whole
 * set runs as one persistent kernel launch per RK stage, nsteps steps as one
 * CUDA graph (the genasis_batch_* calls below are the same engine).  A batch
 * handle takes only the genasis_hydro_batch_* calls, genasis_hydro_status
 * (returns ENONPHYS if any problem met a non-physical state) and
 * genasis_hydro_destroy; the single-mesh calls return EINVAL for it.
 * ------------------------------------------------------------------------- */
int genasis_hydro_batch_create(int nprob, const genasis_hydro_desc *descs, genasis_hydro_t *out);
/* Initial state of problem iprob from FP64 primitives (host or device):
 * rho[ncell], vel[ndim * ncell], p[ncell] in that problem's layout; resets
 * its time to 0. */
int genasis_hydro_batch_set_primitive(genasis_hydro_t h, int iprob, const double *rho, const double *vel,
                                      const double *p);
/* nsteps RK2 steps of every problem (Eqs. RungeKutta1-3), each with its own
 * dt = cfl * dt_CFL (Eq. courantTimeStep) taken on the device; t_end > 0
 * stops each problem exactly at t_end (0: no end time).  Asynchronous. */
int genasis_hydro_batch_run(genasis_hydro_t h, int nsteps, double cfl, double t_end);
/* Conserved state of problem iprob, (ndim + 2) * ncell values in
 * `precision` (GENASIS_FP64 or GENASIS_FP32_MIXED), host or device;
 * synchronises.  get_times stores the nprob problem times (host). */
int genasis_hydro_batch_get_conserved(genasis_hydro_t h, int iprob, void *U, int precision);
int genasis_hydro_batch_get_times(genasis_hydro_t h, double *t);

/* Attach a trained flux-correction network to a 2D GENASIS_FP32_MIXED
 * single-mesh handle (HLL or HLLC, n[q] >= 6).  The paper has no learned
 * term: the correction, its features, the flux-corrected-transport limiter
 * and the positivity fallback are those of genasis_learned_* below, added to
 * the face flux of Sec. 3.2 so that the update stays in conservation form.
 *   bf16_weights  host or device pointer to the genasis_mlp_param_count()
 *                 parameters (W1 [64][24], b1 [64], W2 [64][64], b2 [64],
 *                 W3 [4][64], b3 [4]) as BF16 values (uint16 bit patterns,
 *                 the upper half of the FP32 value); copied
 *   bytes         2 * genasis_mlp_param_count(); a NULL pointer with
 *                 bytes = 0 detaches the network (plain scheme again)
 * While a network is attached, genasis_hydro_step and genasis_hydro_advance
 * run the corrected scheme on the handle's state and time (same stream);
 * every other call is unchanged.  Returns EINVAL for another kind of handle
 * or a wrong size. */
int genasis_hydro_set_flux_mlp(genasis_hydro_t h, const void *bf16_weights, size_t bytes);

/* ---------------------------------------------------------------------------
 * Learned flux correction (2D).  Not in the paper: the benchmark adds to the
 * face flux of Sec. 3.2 (HLL or HLLC) a correction predicted by a small network
 * from the six-cell primitive stencil across each face:
 *   features (24): for cells i-3 .. i+2 along the face normal, rho/rho_bar - 1,
 *     v_n/c_bar, v_t/c_bar, p/p_bar - 1 (rho_bar, p_bar: stencil means,
 *     c_bar = sqrt(gamma p_bar / rho_bar), v_n / v_t: normal / transverse
 *     velocity);
 *   network: 24 -> 64 -> 64 -> 4, SiLU activations, BF16 weights and
 *     activations, FP32 accumulation (tensor cores);
 *   correction: output k times the flux scale (rho_bar c_bar, rho_bar c_bar^2,
 *     rho_bar c_bar^2, rho_bar c_bar^3) for (mass, normal momentum, transverse
 *     momentum, energy), added to the face flux, so the update stays in
 *     conservation form (every face flux is shared by its two cells);
 *   limiter: flux-corrected transport keeps every conserved variable within
 *     local bounds of the plain update (genasis_learned_set_fct);
 *   fallback: after each RK stage, a cell whose corrected update has rho <= 0
 *     or p <= 0 makes every face it touches use the plain flux, and the cells
 *     around it are recomputed (one a-posteriori pass).
 * Parameters are one FP32 vector of genasis_mlp_param_count() values:
 * W1 [64][24], b1 [64], W2 [64][64], b2 [64], W3 [4][64], b3 [4].
 * ------------------------------------------------------------------------- */
typedef struct genasis_learned *genasis_learned_t;
typedef struct genasis_mlp_opt *genasis_mlp_opt_t;

/* Number of network parameters (6020). */
int genasis_mlp_param_count(void);

/* Corrected 2D solver: desc as for genasis_hydro_create with ndim = 2,
 * precision GENASIS_FP32_MIXED, n[q] >= 6.  Without parameters (or after
 * set_params(NULL)) it runs the plain scheme. */
int genasis_learned_create(const genasis_hydro_desc *desc, genasis_learned_t *out);
int genasis_learned_destroy(genasis_learned_t l);
/* params: host or device pointer to the FP32 parameter vector, copied. */
int genasis_learned_set_params(genasis_learned_t l, const float *params);
/* Flux-corrected transport (Zalesak 1979) on the correction, on by default:
 * the plain flux is the low-order flux and the correction the antidiffusive
 * flux; each face's correction is scaled by C in [0, 1] so that no conserved
 * variable of a cell leaves the range, over the cell and its face neighbours,
 * of the plain-flux update and of the stage input (enabled = 1 or 0). */
int genasis_learned_set_fct(genasis_learned_t l, int enabled);
/* Bound on the network outputs (face frame, before scaling): each output is
 * clamped to [-ylim, ylim]; INFINITY (the default) means no bound. */
int genasis_learned_set_limit(genasis_learned_t l, float ylim);
/* State in FP32 conserved form (4 planes) or from FP64 primitives, host or
 * device; get_conserved synchronises. */
int genasis_learned_set_primitive(genasis_learned_t l, const double *rho, const double *vel, const double *p);
int genasis_learned_set_conserved(genasis_learned_t l, const float *U);
int genasis_learned_get_conserved(genasis_learned_t l, float *U);
/* nsteps RK2 steps with the device CFL step (as genasis_hydro_advance). */
int genasis_learned_advance(genasis_learned_t l, int nsteps, double cfl, double t_end, double *t_out);
/* One corrected TVD RK2 step with the given dt (> 0, no CFL check), enqueued
 * on the handle's stream without synchronising. */
int genasis_learned_step(genasis_learned_t l, double dt);
/* Cells whose corrected update fell back to the plain flux, cumulative. */
int genasis_learned_fallbacks(genasis_learned_t l, long long *cells);
/* GENASIS_OPT_ONE_LAUNCH: 1 (default) runs genasis_learned_advance and
 * genasis_learned_step as one cooperative kernel launch for all the steps of
 * the call (a persistent grid of CTAs that meet at bounded grid barriers
 * between the phases; a barrier that waits about a second sets the timeout
 * status and ends the launch).  The face, network and cell arithmetic is that
 * of the per-phase launches, so states, dt, time and fallback counts are
 * bitwise the same.  0 keeps the per-phase launches (a CUDA graph per call
 * shape).
 * GENASIS_OPT_MLP_TCGEN05: 0 (default) runs the network on mma.sync
 * fragments held in registers; 1 on the 5th-generation tensor cores
 * (tcgen05.mma, operands in shared memory, FP32 accumulators in tensor
 * memory, 128 faces per MMA tile).  Both accumulate the same BF16 products in
 * FP32 in different orders, so their states agree to rounding; for this
 * 24-64-64-4 network the register-resident form is the faster one.
 * Returns EINVAL for another option or value. */
#define GENASIS_OPT_MLP_TCGEN05 3
int genasis_learned_set_option(genasis_learned_t l, int option, int value);
/* Kernel launches one step takes: 1 when one launch covers all the steps of a
 * call, else the per-phase count (2 + 2 x 8 with a network and FCT). */
int genasis_learned_launches_per_step(genasis_learned_t l);
/* Training support on a periodic mesh, device pointers, compact face order
 * f = (axis * ny + j) * nx + i (face (i, j) of axis 0 lies between cells
 * (i-1, j) and (i, j)):
 *   features: X [2 nx ny][32] BF16 (24 features + zeros), scale [2 nx ny][4];
 *   targets:  T [2 nx ny][4] = face-frame (f_target - f_plain) / scale, with
 *             f_target, f_plain [2][4][ny][nx] FP64 in conserved order. */
int genasis_learned_features(genasis_learned_t l, void *X, float *scale);
int genasis_learned_targets(genasis_learned_t l, const double *f_target, const double *f_plain, const float *scale,
                            float *T);

/* Add weight * (F(U^n) + F(U^n + dt K)) / 2 of the step just taken (the
 * effective RK2 face flux), averaged over the `stride` fine faces of each
 * coarse face, to F [2][4][ny/stride][nx/stride] (FP64, device).  2D
 * GENASIS_FP32_MIXED handles only; call right after a step. */
int genasis_hydro_accumulate_face_flux(genasis_hydro_t h, int stride, double weight, double *F);
/* Conservative restriction of a uniform 2D FP32 state by `factor` into
 * U_coarse [4][ny/factor][nx/factor] (device); synchronises. */
int genasis_hydro_restrict(genasis_hydro_t h, int factor, float *U_coarse);

/* Network on tensor cores (device pointers; stream may be NULL):
 *   forward:  Y [n][4] from X [n][32] BF16 (X and Y 16-byte aligned, else
 *             EINVAL), asynchronous: tcgen05 MMAs with FP32 accumulators in
 *             tensor memory, 128 samples per tile; a tile whose wait for the
 *             tensor cores runs out (about a second) leaves NaN in its rows;
 *   gradient: grad [param_count] of mean((y - T)^2) over n samples x 4
 *             outputs, and optionally the sum of squared errors (*loss). */
int genasis_mlp_forward(const float *params, const void *X, long long n, float *Y, void *stream);
int genasis_mlp_gradient(const float *params, const void *X, const float *T, long long n, float *grad, float *loss,
                         void *stream);
/* Adam (beta 0.9 / 0.999, eps 1e-8) on a device copy of the parameters. */
int genasis_mlp_opt_create(const float *params, void *stream, genasis_mlp_opt_t *out);
int genasis_mlp_opt_destroy(genasis_mlp_opt_t o);
/* One gradient step on the batch (X, T device pointers); *loss_out (host, may
 * be NULL) receives the batch mean squared error before the step. */
int genasis_mlp_opt_step(genasis_mlp_opt_t o, const void *X, const float *T, long long n, float lr, float *loss_out);
int genasis_mlp_opt_get_params(genasis_mlp_opt_t o, float *params);

/* One RK2 step with a caller-given dt, like genasis_hydro_step, for callers
 * that cannot allocate device memory: code whose device memory belongs to a
 * pooling allocator that has already reserved it (a cudaMalloc there fails or
 * fragments the pool), and latency-critical loops that must not allocate after
 * initialisation.  The paper has no counterpart: this is an interface choice.
 *   desc   mesh and solver as for genasis_hydro_create (widths are host
 *          pointers); desc->stream is the stream to run on (NULL = the legacy
 *          default stream).
 *   U_in   device pointer, conserved state U^n in desc->precision
 *          ((ndim + 2) * ncell values, layout as above); not modified.
 *   U_out  device pointer receiving U^{n+1}; must not overlap U_in.
 * No handle is needed and nothing is allocated (no cudaMalloc, cudaFree or
 * allocating library call): the stage buffer, reduction partials, device
 * scalars and geometry tables live in one static 32 MiB device array that
 * every GPU loading the library holds until the process exits.  Limits: at
 * most 4096 cells per axis, (ndim + 2) * ncell * sizeof(element) at most about
 * 31 MiB (for example 1.5 M cells in 3D FP32, 0.78 M in 3D FP64), at most
 * 4096 CTAs per stage; larger sizes return GENASIS_EINVAL with a message.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current and caches it for the life
 * of the process: do not call it on a device after a cudaDeviceReset of that
 * device.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (other streams, other host threads) race on
 * it.  Every call copies the widths from host memory and synchronises the
 * stream, so it cannot be made while that stream is capturing (it returns
 * GENASIS_EINVAL then).  Returns GENASIS_ENONPHYS if the step met a
 * non-physical state. */
int genasis_hydro_step_noalloc(const genasis_hydro_desc *desc, const void *U_in, void *U_out, double dt);

/* ---------------------------------------------------------------------------
 * Batches: many independent 1D and 2D problems of uneven size advanced
 * together.  Every problem follows the same update as a single handle (same
 * equations and passages as above) with its own mesh, boundaries, gamma, time
 * and CFL time step; all problems of a batch share solver, theta and
 * precision.  Each RK stage of the whole batch is one persistent kernel launch
 * whose CTAs take (problem, tile, chunk) work items largest first from a
 * device counter; genasis_batch_run captures nsteps steps as one CUDA graph.
 * Arrays of problem i use the single-handle layout for that problem's ndim
 * and n.  Ownership, pointer kinds, synchronisation and error codes follow the
 * conventions at the top of this file.
 * ------------------------------------------------------------------------- */
typedef struct genasis_batch *genasis_batch_t;

/* One problem: ndim 1 or 2, n[q] >= 2 cells, widths[q] host arrays of n[q]
 * positive widths, bc codes as for genasis_hydro_desc, gamma > 1. */
typedef struct {
  int ndim;
  int n[2];
  const double *widths[2];
  int bc_lo[2];
  int bc_hi[2];
  double gamma;
} genasis_batch_problem;

/* Create a batch of nprob problems (copied); allocates one state arena for
 * all problems and builds the work list.  stream as in genasis_hydro_desc. */
int genasis_batch_create(int nprob, const genasis_batch_problem *probs, int solver, double theta, int precision,
                         void *stream, genasis_batch_t *out);
int genasis_batch_destroy(genasis_batch_t b);

/* Initial state of problem iprob from FP64 primitives (host or device),
 * rho[ncell], vel[ndim * ncell], p[ncell]; resets that problem's time. */
int genasis_batch_set_primitive(genasis_batch_t b, int iprob, const double *rho, const double *vel, const double *p);
/* Conserved state of problem iprob, (ndim + 2) * ncell values in `precision`
 * (host or device); synchronises. */
int genasis_batch_get_conserved(genasis_batch_t b, int iprob, void *U, int precision);

/* nsteps RK2 steps of every problem, each with its own dt = cfl * dt_CFL (taken
 * on the device per problem); t_end > 0 stops each problem exactly at t_end.
 * Asynchronous; one CUDA-graph launch. */
int genasis_batch_run(genasis_batch_t b, int nsteps, double cfl, double t_end);

/* Per-problem times (nprob doubles); synchronises. */
int genasis_batch_get_times(genasis_batch_t b, double *t);
/* Synchronise; GENASIS_ENONPHYS if any problem met a non-physical state, with
 * *first_bad (if non-NULL) set to the lowest such problem index, else -1. */
int genasis_batch_status(genasis_batch_t b, int *first_bad);

/* Tile index (0 .. count-1: 128 or 256 threads per CTA) and rows per 2D work
 * item (0 = automatic).  info[0..6] = (tile, threads, rows per item, work
 * items, persistent CTAs, tile count, total cells / 2^20). */
int genasis_batch_set_tile(genasis_batch_t b, int tile, int chunk);
int genasis_batch_get_tile(genasis_batch_t b, int *info);
/* Time each tile and a few chunk sizes for trial_steps steps on the current
 * state, keep the fastest, restore state and times; cache file as for
 * genasis_hydro_autotune (keyed by problem count, cells, precision, solver). */
int genasis_batch_autotune(genasis_batch_t b, int trial_steps, const char *cache_path);
/* Device durations of the last step's two persistent stage launches and the
 * per-problem dt kernel (ms[0..2]) from one extra profiled step; synchronises. */
int genasis_batch_profile_step(genasis_batch_t b, double cfl, float *ms);

/* ---------------------------------------------------------------------------
 * Multilevel evolution with subcycling on a fixed mesh of nested levels
 * (Sec. 3.7, Algorithms Evolve, EvolveLevel, StepLevel).  The paper refines
 * oct-tree cells inside nested spheres; here each level l >= 1 is an n^d box
 * over the central half of level l-1 (per axis) at twice its resolution, so
 * its cells are the children of the coarse cells [n/4, 3n/4).  Level 0 covers
 * the cube of side `size` with the wall rule `bc` on every face.
 *   - a level l >= 1 is stored with a two-cell exterior ring: (n+4)^d cells,
 *     x fastest; level 0 as n^d;
 *   - before each step of level l the ring is prolonged from level l-1
 *     (coarse value plus minmod-limited conserved slopes times the child
 *     offset) and held through both RK stages;
 *   - after a step, covered coarse cells take the mean of their children,
 *     and the uncovered coarse cells next to a child's box have the coarse
 *     flux through the shared faces replaced by the child's time-integrated
 *     Heun-effective flux (conservation on leaf cells);
 *   - the deepest level steps with cfl x min_l dt_CFL(l) / 2^(L-1-l), each
 *     coarser level by the time its child advanced; between a level's two
 *     steps its parent takes a provisional forward-Euler substep, undone
 *     afterwards.
 * n a multiple of 4 in [16, 1024]; ndim 2 or 3; GENASIS_FP64 or GENASIS_FP32_MIXED;
 * HLL or HLLC. */
typedef struct genasis_fmr *genasis_fmr_t;
typedef struct {
  int ndim;          /* 2 or 3 */
  int n;             /* cells per axis on every level */
  int nlevels;       /* 1 .. 12 */
  double size;       /* side of the level-0 cube */
  int bc;            /* GENASIS_BC_* on every face of level 0 */
  double gamma;
  int solver;        /* GENASIS_HLL or GENASIS_HLLC */
  double theta;      /* limiter parameter */
  int precision;     /* GENASIS_FP64 or GENASIS_FP32_MIXED */
  void *stream;      /* NULL: the library creates one */
} genasis_fmr_desc;

int genasis_fmr_create(const genasis_fmr_desc *desc, genasis_fmr_t *out);
int genasis_fmr_destroy(genasis_fmr_t f);
/* Set / read level `level` in its stored layout (conserved, FP64, host or
 * device; (ndim+2) planes of n^d (level 0) or (n+4)^d cells). */
int genasis_fmr_set_level(genasis_fmr_t f, int level, const double *U);
int genasis_fmr_get_level(genasis_fmr_t f, int level, double *U);
/* nsteps global steps (one pass of Algorithm Evolve's loop each); if t_out
 * is non-NULL it synchronises, stores the time reached and reports
 * ENONPHYS if any level met a non-physical state. */
int genasis_fmr_step(genasis_fmr_t f, int nsteps, double cfl, double *t_out);
/* Autotune each level's launch configuration (genasis_hydro_autotune on the
 * level's mesh and current state, which is restored; trial_steps >= 1).  Call
 * after the levels are set; results are bitwise those of any other
 * configuration.  Synchronises. */
int genasis_fmr_autotune(genasis_fmr_t f, int trial_steps);

#ifdef __cplusplus
}
#endif

#endif /* GENASIS_HYDRO_H */
