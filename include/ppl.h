/*
 * ppl -- GB300-native pseudopotential lattice Boltzmann library for boiling heat transfer.
 *
 * C ABI of the hot path of arXiv 2201.04560 (Jaramillo, Mapelli, Cabezas-Gomez,
 * "Pseudopotential Lattice Boltzmann Method for boiling heat transfer: a mesh refinement
 * procedure"): one fused per-node update of the D2Q9 MRT pseudopotential LBM (Sec. 2,
 * Eqs. lbm, collisionMRT, EquilibriumDistribution, DensityAndVelocityRelationToF), the
 * Peng-Robinson pseudopotential (Eqs. psi, peng-robinson), the Shan-Chen force with the
 * psi-based wall adhesion (Eqs. shanchen, shanchen-walls, psi-based-formula), gravity
 * (Eq. gravitational_force), the Li sigma/kappa source terms (Eqs. li_source_terms, S,
 * surface-tension-correction-term-C/-Q, Q-psi-based), Zou-He wet-node walls and the
 * hybrid finite-difference temperature equation (Eq. energy-equation) advanced by a
 * second-order Runge-Kutta (Heun) step.
 *
 * Conventions
 *  - All values are lattice units. Fields are row-major [ny][nx]: node (x, y) is element
 *    y*nx + x. Populations are [9][ny][nx] in the velocity order of Sec. 2:
 *    c = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *  - Boundary sides are indexed 0 = x-min, 1 = x-max, 2 = y-min, 3 = y-max. At most one
 *    axis may be non-periodic for the hydrodynamics (no wall corners).
 *  - Every entry point returns PPL_OK (0) or a negative PPL_E_* code; nothing throws
 *    across the ABI. ppl_strerror() names a code. Thread safety: one handle must not be
 *    used from two host threads at once; distinct handles are independent.
 *  - Ownership: the library owns all device memory of a handle (freed by ppl_destroy).
 *    Host and device buffers passed in are caller-owned, only read or written during the
 *    call, and must stay valid for its duration. ppl_init copies the configuration,
 *    including the optional per-node boundary arrays.
 *  - Asynchrony: work is enqueued on the handle's stream (default: the legacy default
 *    stream; see ppl_set_stream). ppl_step, ppl_fields*, ppl_norms, ppl_save and
 *    ppl_populations synchronise that stream before they return.
 */
#ifndef PPL_H
#define PPL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define PPL_OK 0
#define PPL_E_INVAL (-1)   /* bad size, parameter or boundary combination; psi undefined at init */
#define PPL_E_CUDA (-2)    /* a CUDA runtime call failed (no device, launch failure, ...) */
#define PPL_E_NUMERIC (-3) /* the device status word reports NaN, rho <= 0 or a negative psi argument */
#define PPL_E_TIMEOUT (-4) /* a bounded device wait ran out */
#define PPL_E_IO (-5)      /* checkpoint file missing, short, or written by another configuration */
#define PPL_E_NOMEM (-6)   /* device or host allocation failed */

/* ---- enumerations ---- */
#define PPL_FP64 0    /* populations and arithmetic in FP64 */
#define PPL_FP32DEV 1 /* FP32 arithmetic; f_i - w_i rho_ref and T - T_ref stored in FP32 */
/* FP64 state that also carries its derivative with respect to sigma (Eq. S) or kappa
 * (Eq. Q): forward-mode (tangent-linear) sensitivity, read with ppl_tangent_fields. The
 * initial state has zero derivative; the derivative of rho_bar of Eq. (gravitational_force)
 * is carried with it (an FP64 domain sum). Not accepted by ppl_step_noalloc, ppl_cross_norm
 * or ppl_wall_heat_flux; ppl_phase_area reads the values. */
#define PPL_FP64_DSIGMA 2
#define PPL_FP64_DKAPPA 3
/* The same in FP32 arithmetic (values stored as f_i - w_i rho_ref and T - T_ref like
 * PPL_FP32DEV, derivatives in FP32; the domain sums and d rho_bar stay FP64). */
#define PPL_FP32_DSIGMA 4
#define PPL_FP32_DKAPPA 5

#define PPL_PERIODIC 0 /* hydrodynamic side kinds */
#define PPL_WALL 1     /* Zou-He no-slip wet node + psi-based adhesion (Sec. 2.2) */
#define PPL_OUTFLOW 2  /* zero-gradient (null Neumann) copy of the first interior line */

#define PPL_T_PERIODIC 0  /* thermal side kinds */
#define PPL_T_DIRICHLET 1 /* boundary nodes held at T_side / T_w */
#define PPL_T_ADIABATIC 2 /* mirror ghost across the wall row (zero normal gradient) */

#define PPL_CONTACT_PSI 0     /* psi-based contact angle model (Eq. psi-based-formula) */
#define PPL_CONTACT_MOD_PSI 1 /* modified psi-based model (Eq. mod-psi-based-formula), constant G_w */

/* status-word bits (ppl_norms.flags) */
#define PPL_FLAG_PSI_NEG 1u /* 2 (p_EOS - rho/3) / G < 0 somewhere: psi undefined */
#define PPL_FLAG_NAN 2u     /* NaN or Inf in rho or T */
#define PPL_FLAG_RHO_NONPOS 4u
#define PPL_FLAG_STALL 8u   /* a staged row copy did not land within the step kernel's wait limit:
                               that step's result is invalid */

/*
 * Simulation configuration (Sec. 2 model parameters; Sec. 3 scaling is applied by the caller).
 *  nx, ny        grid size (nx, ny >= 3; a non-periodic axis needs >= 4 nodes)
 *  precision     PPL_FP64 or PPL_FP32DEV
 *  rho_ref       reference density of the FP32 deviation storage (ignored for FP64)
 *  T_ref         reference temperature: FP32 stores T - T_ref (ignored for FP64)
 *  a, b, R, omega  Peng-Robinson EOS (Eq. peng-robinson); T_c = 0.0778 a / (0.45724 b R)
 *  G             pseudopotential strength of Eq. (psi), must be < 0 (the paper uses -1)
 *  s[9]          diagonal of Lambda in the row order of M: s_rho, s_e, s_zeta, s_j, s_q, s_j, s_q, s_eta, s_eta
 *  eta_l, eta_v  if both > 0, s_eta = 1/(3 eta(rho) + 1/2) per node with eta(rho) linear
 *                between (rho_v, eta_v) and (rho_l, eta_l) (Eq. eta-rho); else s[7], s[8] are used
 *  rho_l, rho_v  anchors of the eta(rho) and lambda(rho) interpolations (rho_l != rho_v)
 *  sigma, kappa  Li thermodynamic-consistency and surface-tension parameters (Eqs. S, Q)
 *  gx, gy        gravity of Eq. (gravitational_force), F^b = g (rho - rho_bar)
 *  cv, lambda_l, lambda_v   energy equation (Eq. energy-equation), lambda linear in rho
 *  energy_on     0: temperature frozen; 1: advanced from step iso_steps on
 *  hydro_bc[4], thermal_bc[4]  side kinds (PPL_PERIODIC.. and PPL_T_PERIODIC..)
 *  T_side[4]     Dirichlet temperature per side; rho_w_side[4] wall density per side
 *  rho_w[4], T_w[4], T_dirichlet[4]  optional per-boundary-node arrays (length ny for
 *                sides 0/1, nx for sides 2/3; NULL = use the per-side value). T_dirichlet
 *                marks each node Dirichlet (1) or adiabatic (0) on a wall side. At corners
 *                the y-sides decide the thermal kind and value.
 *  contact_model PPL_CONTACT_PSI: solid links carry psi(rho_w, T) in F^m and Q (Eqs.
 *                psi-based-formula, Q-psi-based). PPL_CONTACT_MOD_PSI: F^ads = -G_w psi^2
 *                sum_solid w_i c_i and Q drops the solid links (Eqs. mod-psi-based-formula,
 *                Q-mod-psi-based); rho_w is then unused. G_w: finite, used by MOD_PSI only.
 */
typedef struct ppl_config {
  int32_t nx, ny;
  int32_t precision;
  double rho_ref;
  double T_ref;
  double a, b, R, omega, G;
  double s[9];
  double eta_l, eta_v, rho_l, rho_v;
  double sigma, kappa, gx, gy, cv, lambda_l, lambda_v;
  int32_t energy_on;
  int64_t iso_steps;
  int32_t hydro_bc[4], thermal_bc[4];
  double T_side[4];
  double rho_w_side[4];
  const double *rho_w[4];
  const double *T_w[4];
  const uint8_t *T_dirichlet[4];
  int32_t contact_model;
  double G_w;
} ppl_config;

/* FP64 diagnostics of the current state (the denominators of the space-time norms of
 * Eqs. rel-diff-timestep and global-rel-diff are sum_abs_rho and sum_abs_T). */
typedef struct ppl_norms_t {
  int64_t step;
  double mass;     /* sum of rho over all nodes */
  double rho_mean; /* mass / (nx ny): the rho_bar of the next step's F^b */
  double sum_abs_rho, sum_abs_T;
  double rho_min, rho_max, T_min, T_max;
  uint32_t flags; /* PPL_FLAG_* accumulated since init */
} ppl_norms_t;

typedef struct ppl_sim ppl_t;
typedef struct ppl_batch ppl_batch_t; /* a set of handles stepped together (ppl_batch_create) */

/* Allocate device state and initialise it: f = f^eq(rho0, u0) (Eq. EquilibriumDistribution),
 * T = T0; Dirichlet nodes take their wall value and an outflow line copies the first
 * interior line. rho0, ux0, uy0, T0: host FP64 [ny][nx]. Returns PPL_E_INVAL for bad
 * sizes or parameters, or when psi is undefined (Eq. psi) anywhere in the initial state.
 * On success *out owns the handle (release with ppl_destroy). */
int ppl_init(const ppl_config *cfg, const double *rho0, const double *ux0, const double *uy0,
             const double *T0, ppl_t **out);

/* Re-initialise the state of an existing handle from host fields (as ppl_init, no
 * allocation); the step counter restarts at 0. */
int ppl_reset(ppl_t *h, const double *rho0, const double *ux0, const double *uy0, const double *T0);

/* Enqueue all further work of h on `cuda_stream` (a cudaStream_t, e.g. a PyTorch stream's
 * handle; NULL = legacy default stream). The stream must outlive its use by h. */
int ppl_set_stream(ppl_t *h, void *cuda_stream);

/* Advance nsteps >= 0 time steps (one fused kernel launch per step, replayed from CUDA
 * graphs of 32, 16, 8, 4 and 2 steps, at most one step launched on its own), then
 * synchronise the stream and check the device status word: PPL_E_NUMERIC if any flag is
 * set. The first call that can use a graph captures all of them (for the current energy
 * setting), so that call takes longer. Inside a stream capture of the caller's, steps are
 * launched one by one into that capture. */
int ppl_step(ppl_t *h, int64_t nsteps);

/* As ppl_step but returns right after enqueueing; no status check, no synchronisation. */
int ppl_step_async(ppl_t *h, int64_t nsteps);

/* Synchronise the stream and check the status word (pairs with ppl_step_async). */
int ppl_sync(ppl_t *h);

/* Macroscopic fields of the current state into caller-owned host FP64 [ny][nx] buffers:
 * rho, u = (sum_i f_i c_i + F/2)/rho (Eq. DensityAndVelocityRelationToF) and T. Any
 * pointer may be NULL to skip that field. */
int ppl_fields(ppl_t *h, double *rho, double *ux, double *uy, double *T);

/* As ppl_fields into caller-owned DEVICE buffers (e.g. torch data_ptr()s), each [ny][nx]
 * of dtype 0 = FP64 or 1 = FP32; written on the handle's stream, synchronised on return. */
int ppl_fields_device(ppl_t *h, void *rho, void *ux, void *uy, void *T, int dtype);

/* Populations of the current state (post-streaming, boundary conditions applied) as host
 * FP64 [9][ny][nx], decoded from the FP32 deviation storage when precision is FP32DEV. */
int ppl_populations(ppl_t *h, double *f);

/* The current state as FP64 device arrays: absolute populations f [9][ny][nx] (decoded
 * from the FP32 deviation storage when precision is FP32DEV) and T [ny][nx], written into
 * caller-owned device buffers (no allocation). The input of the adjoint sweep
 * (ppl_adjoint_step). PPL_E_INVAL for sensitivity handles or NULL buffers. Synchronises. */
int ppl_state_device(ppl_t *h, double *f, double *T);

/* Device snapshot of the stored state (f, T and the step statistics in the working
 * precision, exactly as the step kernel reads them), for checkpointed recomputation: the
 * adjoint sweep restores a snapshot and steps forward again, bit-identically.
 * ppl_snapshot_bytes: size of one snapshot (0 for NULL). ppl_snapshot copies into the
 * caller's device buffer dst, ppl_restore copies src back and sets the step counter (which
 * decides when the energy equation starts, iso_steps). Both are enqueued on the handle's
 * stream and do not synchronise; dst / src stay caller-owned. */
size_t ppl_snapshot_bytes(const ppl_t *h);
int ppl_snapshot(ppl_t *h, void *dst);
int ppl_restore(ppl_t *h, const void *src, int64_t step);

/* Derivatives d rho, d u_x, d u_y, d T of the current state with respect to the parameter
 * of a sensitivity handle (PPL_FP64_D* or PPL_FP32_D*), as host FP64 [ny][nx] arrays (NULL
 * pointers skip a field). PPL_E_INVAL for other handles. Synchronises. */
int ppl_tangent_fields(ppl_t *h, double *drho, double *dux, double *duy, double *dT);

/* FP64 diagnostics of the current state; synchronises. */
int ppl_norms(ppl_t *h, ppl_norms_t *out);

/* Checkpoint: write / restore the full state (populations, T, rho_bar, step counter) with
 * a header carrying the grid, precision and a hash of the configuration. ppl_load on a
 * handle with a different configuration returns PPL_E_IO. A resumed run is bit-identical
 * to an uninterrupted one. */
int ppl_save(ppl_t *h, const char *path);
int ppl_load(ppl_t *h, const char *path);

/* Number of fused step kernels launched by this handle since init (for launch accounting). */
int64_t ppl_launch_count(const ppl_t *h);

/* Release the handle and its device memory (NULL is ignored). */
void ppl_destroy(ppl_t *h);

/*
 * One time step on caller-owned device buffers, with no device memory allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- host applications or plugins whose framework owns and pre-plans every
 * device allocation, and latency-critical loops where an allocation's implicit device
 * synchronisation is not acceptable. It runs the same fused step kernel as ppl_step.
 *
 *  cfg        configuration as for ppl_init; energy_on selects whether T is advanced in
 *             this step (iso_steps is not used). Per-boundary-node arrays (rho_w, T_w,
 *             T_dirichlet) are not supported here: they would need device copies.
 *  f_in, T_in    device state in: populations [9][ny][nx] and T [ny][nx], doubles for
 *             PPL_FP64, floats holding f_i - w_i rho_ref and T - T_ref for PPL_FP32DEV;
 *             each pointer 8-byte aligned
 *  f_out, T_out  device state out, same layout and alignment; neither may overlap any
 *             other of the four buffers (the step reads the neighbours of what it writes).
 *             A line on an OUTFLOW side (x = nx-1 or x = 0, y likewise) is never written:
 *             the step treats it as a copy of the first interior line and reads that line
 *             instead, so the caller's outflow line keeps whatever it held before the call.
 *             A caller that needs it copies the first interior line there.
 *  stats_in   device double[1]: rho_bar (mean density) of the input state
 *  stats_out  device double[2]: rho_bar and total mass of the output state
 *  status     device uint32: PPL_FLAG_* bits are OR-ed in (the caller clears it)
 *  cuda_stream   stream to enqueue on (NULL: legacy default stream); nothing synchronises
 *
 * Scratch: the FP64 per-CTA partials of the mass reduction and a completion counter live
 * in a static device array of the library (4096 partials, 32 KB), held by every GPU that
 * loads the library until the process exits. A launch grid of more than 4096 CTAs (the
 * default shape is one wave of resident CTAs, so only very wide grids, beyond about 4096
 * column strips of 120-122 columns, reach it) is rejected with PPL_E_NOMEM before anything
 * runs (the configuration is checked before the buffer pointers); the sensitivity
 * precisions, null, misaligned or overlapping buffers with PPL_E_INVAL.
 * The first call on each device resolves the scratch's device address and sets kernel
 * attributes; make that first call before any stream capture. That set-up is kept for the
 * life of the process: after cudaDeviceReset on a device the library must not be called
 * on that device again (the resolved address would be stale). All calls share the one scratch array and it keeps the last
 * call's contents (the counter is cleared by each call): calls that overlap on the GPU,
 * on different streams or threads, race and must be serialised by the caller.
 * Returns PPL_OK, PPL_E_INVAL (bad arguments, unsupported per-node arrays), PPL_E_NOMEM
 * (a grid beyond the static scratch) or PPL_E_CUDA.
 */
int ppl_step_noalloc(const ppl_config *cfg, const void *f_in, const void *T_in, void *f_out, void *T_out,
                     const double *stats_in, double *stats_out, uint32_t *status, void *cuda_stream);

/* Static description of a return code. */
const char *ppl_strerror(int code);

/*
 * Reverse-mode (adjoint) sweep of one fused step, for the sigma / kappa calibration of
 * Sec. 3.2 (Eqs. integral_coexistence_curve, surface_tension: sigma and kappa tuned per
 * mesh) done on the lattice by gradient descent. For a scalar J of the state after the
 * step, with fbar_in = dJ/df^{n+1}, it writes fbar_out = (df^{n+1}/df^n)^T fbar_in and adds
 * (df^{n+1}/d sigma, df^{n+1}/d kappa)^T fbar_in to grad[0], grad[1] (FP64). The step is the
 * one of Sec. 2 (Eqs. psi, peng-robinson, shanchen, Q, DensityAndVelocityRelationToF,
 * collisionMRT, S, C, lbm) on the boxes the calibration uses: every side periodic,
 * isothermal (energy_on = 0), no gravity, constant relaxation rates (eta_l, eta_v unset);
 * other configurations return PPL_E_INVAL.
 *
 *  cfg        configuration of the forward step (sigma, kappa, rates, EOS)
 *  f, T       device FP64 state of the step's input: absolute populations [9][ny][nx]
 *             and T [ny][nx] (ppl_state_device gives them for any handle precision)
 *  fbar_in    device FP64 [9][ny][nx]: dJ/df of the step's output
 *  fbar_out   device FP64 [9][ny][nx]: dJ/df of the step's input; must not be fbar_in
 *  grad       device FP64 [2], accumulated (+=) in a fixed order: bitwise reproducible
 *  scratch    device workspace of ppl_adjoint_scratch_bytes(nx, ny) bytes, caller-owned
 *  cuda_stream   stream to enqueue on (NULL: legacy default stream); nothing synchronises
 * Returns PPL_OK, PPL_E_INVAL or PPL_E_CUDA.
 */
size_t ppl_adjoint_scratch_bytes(int32_t nx, int32_t ny);
int ppl_adjoint_step(const ppl_config *cfg, const double *f, const double *T, const double *fbar_in,
                     double *fbar_out, double *grad, void *scratch, void *cuda_stream);

/* ---- host helpers of the refinement procedure (Sec. 3), FP64 ---- */

/* Critical temperature of the Peng-Robinson EOS: T_c = 0.0778 a / (0.45724 b R) (Sec. 2.1). */
double ppl_tc(double a, double b, double R);

/* Maxwell equal-area coexistence of the PR isotherm at T < T_c (the target of the sigma
 * tuning of Sec. 3.2): writes rho_v, rho_l and p_sat. PPL_E_INVAL if T >= T_c or on bad
 * parameters. */
int ppl_maxwell(double a, double b, double R, double omega, double T, double *rho_v,
                double *rho_l, double *p_sat);

/* Peng-Robinson pressure of Eq. (peng-robinson) at (rho, T) and its derivative dp/drho at
 * fixed T (any T > 0, including supercritical). PPL_E_INVAL outside b rho < 1. Host only. */
int ppl_pressure(double a, double b, double R, double omega, double T, double rho, double *p, double *dp_drho);

/* Eq. (a-deltax): a on a mesh of n nodes per length, from a_base on n_base nodes. */
double ppl_refine_a(double a_base, int32_t n_base, int32_t n);

/* Sec. 3.2 step 2: the sigma for which the mechanical-stability coexistence of Eq.
 * (integral_coexistence_curve) lands on the Maxwell densities at temperature T (secant
 * started at -16 G sigma_0 = 2). PPL_E_INVAL for T >= T_c, bad parameters or no convergence. */
int ppl_sigma_for(double a, double b, double R, double omega, double G, double T, double *sigma);

/* Planar surface tension of Eq. (surface_tension) at (T, sigma, kappa): the profile solves the
 * constant normal stress of the Sec. 2.1 pressure tensor (the (1 - kappa) term read as
 * psi grad grad psi) between the mechanical-stability coexistence densities. */
int ppl_gamma_planar(double a, double b, double R, double omega, double G, double T, double sigma, double kappa,
                     double *gamma);

/* Sec. 3.2 step 3, Eq. (gamma-meshes-relation) with 0 = the base mesh: the kappa of a mesh
 * with n nodes per length such that gamma scales with dx (gamma_n = gamma_base n_base / n);
 * a follows Eq. (a-deltax), sigma is tuned on each mesh, T = T_ratio T_c on each mesh. */
int ppl_kappa_for(double a_base, int32_t n_base, int32_t n, double b, double R, double omega, double G,
                  double T_ratio, double kappa_base, double *kappa);

/* The refinement procedure of Sec. 3 applied to a configuration: grid x n/n_base; a per
 * Eq. (a-deltax); temperatures (T_side, T_ref) with T_c (~ dx^2); gravity ~ dx^3 (Table 1);
 * sigma tuned at T_ratio T_c; kappa per Eq. (gamma-meshes-relation). lambda, c_v, eta, rho_w
 * and the MRT rates are O(1) and kept. The time step scales as dx^2: one base step is
 * (n / n_base)^2 refined steps, and iso_steps is scaled by that factor. Per-boundary-node arrays must be rebuilt by the caller
 * (PPL_E_INVAL if base has any). */
int ppl_refine(const ppl_config *base, int32_t n_base, int32_t n, double T_ratio, ppl_config *out);

/* ---- mesh refinement sequence (Sec. 3, Sec. 4.1-4.3) ---- */

/* Cross-grid difference of Eqs. (rel-diff-timestep) and (global-rel-diff): the field of
 * `coarse` is interpolated bilinearly onto every node of `fine` and
 *   *num = sum_fine |I(coarse) - fine|,   *den = sum_fine |fine|        (FP64 sums),
 * so num/den is the relative L1 difference of the two meshes and sum over several output
 * times of num / sum of den is the global one. field: 0 = rho, 1 = the reduced temperature
 * T / T_c of each mesh (T_c ~ a scales with dx^2 under Table 1's refinement). The two handles
 * cover the same physical domain with the same hydrodynamic sides (PPL_E_INVAL
 * otherwise); their sizes are arbitrary. Coordinates map cell-centred on periodic axes
 * (fine line g sits at coarse (g + 1/2) nc/nf - 1/2, wrapping) and node-aligned on bounded
 * axes (g (nc - 1)/(nf - 1), end lines on end lines). Outflow lines read their copied
 * first interior line, as everywhere in this library. Reads the current state of both
 * handles (after all work queued on both streams); synchronises; temporary device memory
 * is allocated and freed inside the call. */
int ppl_cross_norm(const ppl_t *coarse, const ppl_t *fine, int field, double *num, double *den);

/* A batch of n (1..64) distinct handles advanced together: one outer step advances
 * handle k by substeps[k] >= 1 steps (with dt ~ dx^2 a refinement sequence dx, dx/2, dx/4
 * takes 1, 4, 16). The handles' grids run concurrently, as the branches of one CUDA graph
 * per outer step (two outer steps when a substep count is odd, so that every ping-pong
 * buffer returns to its slot); the graph is captured on first use and re-captured only
 * when the isothermal/energy pattern changes (cfg.iso_steps) or a handle's launch shape
 * changed (ppl_set_launch, ppl_autotune). Results are identical, bit for bit, to calling
 * ppl_step(h_k, outer * substeps[k]) on each handle. The handles stay owned by the caller
 * and must outlive the batch; the batch owns its own streams. */
int ppl_batch_create(ppl_t *const *sims, const int32_t *substeps, int32_t n, ppl_batch_t **out);
/* Advance every handle of the batch by `outer` outer steps; the work is ordered after
 * everything already queued on the handles' streams, and those streams continue after it.
 * Synchronises and returns the first non-OK status of the handles (PPL_E_NUMERIC). */
int ppl_batch_step(ppl_batch_t *b, int64_t outer);
void ppl_batch_destroy(ppl_batch_t *b);

/* How a batch runs its outer steps (Sec. 3 refinement sequence, dt ~ dx^2).
 * PPL_BATCH_GRAPH: one CUDA graph per outer step whose concurrent branches
 * launch each handle's steps. PPL_BATCH_PERSISTENT: one persistent launch per ppl_batch_step
 * call, captured in a CUDA graph, for handles that all step with the FP32 two-column kernel
 * (PPL_E_INVAL otherwise): resident CTAs take the tiles of every mesh's steps in time order
 * from a ticket counter, each tile waiting until the previous step of its mesh is complete;
 * results are bitwise those of stepping each handle by itself. Every such wait gives up
 * after the batch's wait limit (default 1 s, ppl_batch_set_wait_limit, in ns); a wait that
 * ran out stops the launch, sets PPL_FLAG_STALL in the handle's status word and makes
 * ppl_batch_step return PPL_E_TIMEOUT, after which the handles' states are undefined
 * (ppl_reset or ppl_load them). ppl_launch_count counts the steps a handle made. */
#define PPL_BATCH_GRAPH 0
#define PPL_BATCH_PERSISTENT 1
#define PPL_BATCH_AUTO 2 /* the default: persistent where it applies and no handle has gravity, else graph */
int ppl_batch_set_mode(ppl_batch_t *b, int mode);
int ppl_batch_get_mode(const ppl_batch_t *b);
int ppl_batch_set_wait_limit(ppl_batch_t *b, int64_t ns);

/* Liquid area of the current state for the droplet radius R(t) of Sec. 4.1:
 *   *area = sum over the nodes of clamp((rho - rho_lo) / (rho_hi - rho_lo), 0, 1)   (FP64),
 * a volume-fraction count in lattice nodes (R = sqrt(area / pi) for one droplet). Outflow
 * lines count their copied first interior line. rho_hi > rho_lo (PPL_E_INVAL otherwise);
 * runs after all work queued on the handle's stream and synchronises it. */
int ppl_phase_area(ppl_t *h, double rho_lo, double rho_hi, double *area);

/* Eq. (relative-change-R): *out = sum_i |R[i] - R_star[i]| / sum_i |R_star[i]| over n >= 1
 * samples of two series taken at the same physical times (R_star on the finer mesh, both in
 * the same length unit). Host only. PPL_E_INVAL for n < 1 or an all-zero R_star. */
int ppl_relative_change(const double *R, const double *R_star, int64_t n, double *out);

/* Eq. (pool-heat-flux): mean conductive heat flux entering the domain through boundary
 * line `side` (0 = x-min, 1 = x-max, 2 = y-min, 3 = y-max),
 *   *q = (1/L) sum over the L nodes of the line of -lambda(rho) dT/dn,
 * n the inward normal, dT/dn = (-3 T_0 + 4 T_1 - T_2) / 2 from the line and the next two
 * lines inward (second-order one-sided), lambda(rho) linear between (rho_v, lambda_v) and
 * (rho_l, lambda_l) as in the energy equation. Positive when heat enters the fluid.
 * PPL_E_INVAL for a side with neither a hydrodynamic nor a thermal boundary, or fewer than
 * 3 lines across. Synchronises the handle's stream. */
int ppl_wall_heat_flux(ppl_t *h, int side, double *q);

/* Time shift of Eq. (rel-diff-minimize): with `coarse` at time tau - m (its own steps) and
 * `finest` at tau, evaluates sum_fine |I(theta^coarse) - theta^finest| (the numerator of
 * ppl_cross_norm) at the shifts delta = -m, -m + stride, ..., <= m, stepping `coarse` by
 * `stride` between evaluations, and returns the minimising shift in *delta (coarse steps)
 * and the minimum in *num_min (may be NULL). `coarse` is left at the last shift evaluated.
 * field: 0 = rho, 1 = T. m >= 0, stride >= 1; same hydrodynamic sides (PPL_E_INVAL).
 * Synchronises both handles' streams. */
int ppl_time_shift(ppl_t *coarse, const ppl_t *finest, int field, int64_t m, int64_t stride, int64_t *delta,
                   double *num_min);

/* Contact angle (degrees, measured through the liquid) of one droplet on boundary line
 * `side` of a host density field rho[ny][nx] (e.g. from ppl_fields), read as a circular cap
 * (Sec. 4.3.1 contact-angle tests). The base is the first line from the wall inward (within
 * half the domain) whose densest node exceeds rho_mid with a crossing of rho = rho_mid on
 * each side; from its half-width a, its distance n0 from the wall and the crossing h along
 * the inward line through the base centre, the circle through (+-a, n0) and (0, h) gives
 * theta = 90 deg + asin(yc / Rc), clamped to [0, 180] (yc: height of its centre above the
 * wall line; a droplet that left the wall reads 180). Crossings by linear interpolation.
 * Host only. PPL_E_INVAL when no base or top is found (e.g. a film over the whole wall). */
int ppl_contact_angle(const double *rho, int32_t nx, int32_t ny, int side, double rho_mid, double *theta);

/* ---- launch shape ---- */

/* Rows per CTA of the fused step kernel (the grid is strips of columns x ceil(ny / rows)
 * row blocks; every CTA recomputes 6 halo rows). rows = 0 restores the default: one wave
 * of resident CTAs over the rows, except for the two-column FP32 step on a grid whose wave
 * would have blocks of 28 rows or more: there one wave of blocks of ~0.86 ny / wave rows
 * covers the lower part and blocks of ~0.27 times that height the rest, so that CTAs
 * freed early take short blocks and the SMs stay full until the step ends.
 * 1 <= rows <= ny otherwise (PPL_E_INVAL; uniform blocks). Results do not depend on the shape except
 * through the rounding of the domain-mass sum of Eq. (gravitational_force), which is
 * summed per CTA (last-bit differences of rho_bar where gravity is on). Drops the
 * handle's captured graphs; synchronises. */
int ppl_set_launch(ppl_t *h, int32_t rows_per_cta);

/* Step kernel of an FP32 handle. PPL_KERNEL_COLUMN: one column per thread (any
 * boundaries). PPL_KERNEL_PAIR: two adjacent columns per thread with packed f32x2
 * arithmetic, for domains hydrodynamically periodic in x with an even nx (PPL_E_INVAL
 * otherwise; the temperature may be held on the x lines). PPL_KERNEL_AUTO (the default at ppl_init): PAIR
 * where it applies, else COLUMN. FP64 and tangent handles always use the one-column
 * kernel. Resets the launch shape to its default and drops captured graphs; synchronises.
 * ppl_get_kernel returns the kernel in use. */
#define PPL_KERNEL_AUTO 0
#define PPL_KERNEL_COLUMN 1
#define PPL_KERNEL_PAIR 2
int ppl_select_kernel(ppl_t *h, int kernel);
int ppl_get_kernel(const ppl_t *h);
/* Launch shape in use: rows of the (first) row blocks and CTAs per step launch. */
int ppl_get_launch(const ppl_t *h, int32_t *rows_per_cta, int32_t *ctas);
/* 1 if the two-column FP32 step stages rows by TMA (tensor maps of the state were encoded at
 * ppl_init: FP32, nx a multiple of 4 and at least one strip wide), 0 if every strip uses
 * per-thread row copies; strips that wrap across the periodic x seam always use the latter. */
int ppl_tma_staging(const ppl_t *h);

/* Check of the step kernel's bounded waits: launches one CTA on the current device that waits,
 * with the wait used for TMA-staged rows, on an mbarrier that nothing completes, for limit_ns
 * (1 .. 1e9), and stores the status word it leaves in *flags (PPL_FLAG_STALL expected). The
 * context stays usable. Synchronous; PPL_E_INVAL for a limit out of range or a NULL flags. */
int ppl_stall_probe(int64_t limit_ns, uint32_t *flags);

/* Measured FP64 fused-multiply-add rate of the current device: a loop of independent DFMA
 * chains on every SM (4 CTAs x 256 threads per SM, iters x 128 DFMAs per thread, 1 <= iters
 * <= 1e6), timed with CUDA events after a warm-up; *dfma_per_s receives the FP64 FMA
 * thread-operations per second (the FP64 step's roofline denominator). Synchronous, on a
 * private stream; PPL_E_INVAL for iters out of range or a NULL result. */
int ppl_fp64_rate(int32_t iters, double *dfma_per_s);

/* Times `steps` (>= 1) steps at each candidate rows-per-CTA (the default and 1..256), for
 * each applicable step kernel (ppl_select_kernel), with CUDA events on the handle's
 * stream, keeps the fastest pair, and restores the state, step
 * counter and launch count it found (the state is copied aside into temporary device
 * memory). *best_rows / *best_ms (may be NULL) receive the choice and its time per step.
 * PPL_E_NUMERIC if the handle's status already reports a numerical failure. */
int ppl_autotune(ppl_t *h, int32_t steps, int32_t *best_rows, double *best_ms);

#ifdef __cplusplus
}
#endif
#endif /* PPL_H */
