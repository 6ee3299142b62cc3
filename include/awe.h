/*
 * awe.h -- C ABI of the GB300 ADER-WENO zone update for the compressible
 * Euler equations (libawe.so, sm_103a).
 *
 * The library performs the per-zone space-time update of the paper's CFD
 * code (Subramanian, Balsara, Bhoriya, Kumar, "Techniques, Tricks and
 * Algorithms for Efficient GPU-Based Processing of Higher Order Hyperbolic
 * PDEs", Sec. II.2, Figs. 1-7): WENO reconstruction of the conserved
 * variables into modal polynomials (Limiter, Fig. 3), an ADER predictor that
 * extends them in time (Predictor, Fig. 4), HLLC Riemann fluxes at
 * space-time quadrature points of every face (Make_Flux_X/Y/Z, Fig. 5), the
 * conservative update (Make_dU_dt, Fig. 6) and the CFL reduction of the next
 * time step (Update_U_Timestep, Fig. 7).  Per grid it also offers the paper's
 * own second-order scheme (order 2), the HLL, HLLEM and Rusanov solvers in
 * place of HLLC (Sec. I.1), and the Runge-Kutta time stepping that Table IV
 * compares ADER with (AWE_SCHEME_SSPRK).  The state stays resident in device
 * memory between steps (the paper's U_skinny lesson, Sec. II.2, Tables I-II);
 * it crosses to the host only through awe_set_state / awe_get_state.
 *
 * Conventions (all entry points):
 *  - Every call returns an awe_status (0 = AWE_OK); nothing aborts or throws
 *    across the ABI.  awe_last_error() gives a message for the last failure
 *    of a handle (valid until the next call on it).
 *  - All device work runs on the CUDA stream given to awe_create (NULL = the
 *    legacy default stream).  Calls that return host scalars synchronise that
 *    stream before returning; the others only enqueue work.
 *  - The library owns all of its device memory (allocated in awe_create,
 *    freed in awe_destroy).  Caller buffers are only read or written during
 *    the call; the library never keeps a caller pointer.
 *  - State layout: conserved variables (rho, rho*v_x, rho*v_y[, rho*v_z], E),
 *    FP64, structure of arrays [var][z][y][x], x fastest, active zones only
 *    (no ghosts); nvar = dim + 2; in 2D the z extent is 1.
 *  - A handle is not thread safe; distinct handles are independent.
 */
#ifndef AWE_H
#define AWE_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct awe_grid awe_grid;

typedef enum {
  AWE_OK = 0,
  AWE_ERR_ARG = -1,          /* invalid argument or configuration */
  AWE_ERR_CUDA = -2,         /* a CUDA call failed (message in awe_last_error) */
  AWE_ERR_OOM = -3,          /* device allocation failed */
  AWE_ERR_NONPHYSICAL = -4,  /* the updated state has rho<=0, p<=0 or a non-finite value */
  AWE_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up */
  AWE_ERR_STATE = -6         /* call out of order (e.g. gate used without weights) */
} awe_status;

/* Boundary conditions, per face (x-low, x-high, y-low, y-high, z-low, z-high).
 * Ghost zones are filled dimension after dimension (x, then y, then z). */
typedef enum {
  AWE_BC_PERIODIC = 0,
  AWE_BC_OUTFLOW = 1,     /* copy of the nearest active zone */
  AWE_BC_REFLECT = 2,     /* mirror image, normal momentum negated */
  AWE_BC_INFLOW = 3,      /* fixed conserved state inflow[face] */
  AWE_BC_DMR_BOTTOM = 4,  /* inflow[face] for x < 1/6, reflecting wall beyond */
  AWE_BC_DMR_TOP = 5,     /* inflow[face] if x < 1/6 + (1 + 20 t)/sqrt(3), else pre */
  AWE_BC_EXCHANGE = 6     /* ghost planes written by the caller with awe_halo_unpack
                             (the neighbour subdomain's planes of a slab
                             decomposition); allowed only on the two faces of the
                             outermost dimension (z in 3D, y in 2D) */
} awe_bc;

/* Arithmetic forms of the step. */
typedef enum {
  AWE_FP64 = 0,       /* every stage in FP64 */
  AWE_FP32_BULK = 1   /* reconstruction, predictor and Riemann fluxes in FP32;
                         the WENO epsilon path (eps + beta_k), the differences
                         of the zone means, the conserved-variable update and
                         the CFL reduction in FP64; the weights formed from
                         eps + beta_k in FP32 */
} awe_prec;

/* Riemann solvers of the corrector (Sec. I.1 names HLLC, HLL, HLLEM and
 * Rusanov).  All use the same face and time quadrature.  HLL, HLLC and HLLEM
 * take Davis-Einfeldt wave speeds from Roe averages; HLLEM restores the
 * contact and shear waves of HLL with the anti-diffusion coefficient
 * 1 - min(u~,0)/S_L - max(u~,0)/S_R; Rusanov's speed is
 * max(|u_L| + c_L, |u_R| + c_R). */
typedef enum {
  AWE_RS_HLLC = 0,
  AWE_RS_HLL = 1,
  AWE_RS_HLLEM = 2,
  AWE_RS_RUSANOV = 3
} awe_riemann;

/* Time stepping.  ADER: the paper's one-step predictor-corrector.  SSPRK: the
 * Runge-Kutta comparison scheme of Table IV (method of lines with the same
 * reconstruction and Riemann fluxes, face fluxes averaged over the face
 * Gauss points only): SSP(2,2), SSP(3,3) or Spiteri and Ruuth's five-stage
 * SSP(5,4) in Shu-Osher form, stage boundary values at t + c_i dt.  The
 * probes (awe_probe_*) cover the ADER path only. */
typedef enum {
  AWE_SCHEME_ADER = 0,
  AWE_SCHEME_SSPRK = 1
} awe_scheme;

typedef struct {
  int dim;               /* 2 or 3 */
  int n[3];              /* active zones per dimension (n[2] ignored in 2D) */
  double lo[3], hi[3];   /* domain box (lo[2], hi[2] ignored in 2D) */
  int order;             /* 2, 3 or 4 (polynomial degree N = order - 1; order 2
                            is the paper's own scheme: MC-limited slopes of
                            Fig. 3, one predictor sweep, one face point) */
  double gamma;          /* ratio of specific heats, ideal gas */
  int bc[6];             /* awe_bc per face */
  double inflow[6][5];   /* conserved state per face (AWE_BC_INFLOW / DMR post-shock) */
  double pre[5];         /* DMR pre-shock conserved state (AWE_BC_DMR_TOP) */
  int prec;              /* awe_prec */
  int picard;            /* predictor sweeps K (0 -> order - 1) */
  double weno_eps;       /* WENO epsilon (absolute), e.g. 1e-12 */
  double lin[4];         /* linear weights of the order candidate stencils */
  double cfl;            /* CFL number used for dt_next */
  int gate;              /* 1: reconstruct unflagged zones with linear weights
                            (troubled-zone gate); needs awe_gate_set_weights */
  int slab;              /* z zones per slab of the intermediate buffers
                            (3D; 0 = whole domain in one slab) */
  int fallback;          /* positivity fallback (not in the paper).  1: a zone
                            whose face states have rho <= 0, p <= 0 or a
                            non-finite value uses its zone mean as every face
                            state (first order).  2 (ADER, no exchanged faces):
                            that, and after the update a zone whose new mean is
                            not physical, with every zone sharing a face with
                            it, is updated again from the old state with the
                            Riemann flux between the two old zone means on each
                            face of a flagged zone (first order, conservative);
                            4 passes, flags accumulating */
  int riemann;           /* awe_riemann: the corrector's Riemann solver */
  int scheme;            /* awe_scheme: ADER (default) or SSP Runge-Kutta */
  int rk_stages;         /* AWE_SCHEME_SSPRK: 2, 3 or 5 stages (0: 2, 3, 5 at
                            orders 2, 3, 4, as in Table IV) */
  double dx[3];          /* zone sizes; 0 = (hi - lo) / n.  A subdomain of a
                            slab decomposition passes the undivided grid's, so
                            that its updates round exactly as that grid's */
} awe_config;

/* Create a grid (allocates all device memory).  Cites: Fig. 1 data region.
 * stream: a cudaStream_t (NULL = default stream).  *out receives the handle.
 * Errors: AWE_ERR_ARG (bad config), AWE_ERR_OOM, AWE_ERR_CUDA. */
int awe_create(const awe_config* cfg, void* stream, awe_grid** out);
/* Destroy a grid and free its device memory (NULL is accepted). */
int awe_destroy(awe_grid* g);
/* Message describing the last failure on this handle ("" if none); a
 * static string if g is NULL (last create failure). */
const char* awe_last_error(const awe_grid* g);

/* Copy a state in (on_device = 0: host pointer, 1: device pointer on this
 * GPU) in the state layout above.  Fig. 1 "update device(U_skinny)".  A
 * page-locked host buffer (cudaHostAlloc / cudaHostRegister) is read directly
 * by the library's scatter kernel; pageable memory is staged through device
 * memory with a copy.  Synchronises when on_device = 0. */
int awe_set_state(awe_grid* g, const double* U, int on_device);
/* Copy the state out (host or device pointer, caller owned).  Fig. 1
 * "update host(U_skinny)".  A page-locked host buffer is written directly by
 * the gather kernel.  Synchronises when on_device = 0. */
int awe_get_state(awe_grid* g, double* U, int on_device);
/* Simulation time t (start of the next step; used by time-dependent BCs). */
int awe_set_time(awe_grid* g, double t);
int awe_get_time(awe_grid* g, double* t);

/* dt = cfl / max over active zones of max_d (|v_d| + c)/dx_d, FP64
 * warp-shuffle max reduction on the current state (Eval_Tstep_Ptwise and
 * REDUCTION(MIN:dt_next), Fig. 7).  The result also becomes the
 * device-resident dt used by awe_step(g, 0, ...).  Synchronises if dt_out. */
int awe_cfl_dt(awe_grid* g, double cfl, double* dt_out);

/* One full step.  ADER (Fig. 1 loop body): ghost zones, reconstruction,
 * predictor, Riemann fluxes (cfg.riemann) with space-time quadrature, FP64
 * update, and the CFL reduction of the updated state.  SSPRK: per stage the
 * ghost zones at the stage time, reconstruction, face values, Riemann fluxes
 * over the face points and the FP64 stage combination; the CFL reduction of
 * the last stage.  dt > 0: use it; dt <= 0: use the
 * device-resident dt (from awe_cfl_dt or the previous step) without any host
 * round trip.  t advances by dt.  dt_next_out (may be NULL, then no
 * synchronisation): cfg.cfl / signal-speed max of the updated state.
 * Returns AWE_ERR_NONPHYSICAL if the updated state is not physical (the
 * state is still updated; only reported when dt_next_out != NULL or by
 * awe_check). */
int awe_step(awe_grid* g, double dt, double* dt_next_out);
/* Synchronise and report a non-physical state flagged by earlier steps. */
int awe_check(awe_grid* g);

/* ---- slab decomposition (one subdomain per grid) ----
 * The paper's code splits the domain into patches and, per time step,
 * exchanges their ghost zones once and takes the MIN of dt over all of them
 * (Sec. II.2, the MPI remarks after Fig. 7; Sec. V, the patch layer): ADER
 * needs one exchange per step, a Runge-Kutta scheme one per stage (Sec. I.1).
 * Here a subdomain is an ordinary grid whose faces towards its neighbours
 * along the outermost dimension have AWE_BC_EXCHANGE.  Before each stage the
 * caller packs the g = order planes next to each such face, moves them to the
 * neighbour (device copy, NCCL, host) and unpacks the neighbour's planes into
 * the ghost planes; the library fills every other ghost zone itself.
 * Buffer layout: [var][plane][inner ghosted extent], planes ordered by
 * increasing coordinate, inner extent (n_y + 2g)(n_x + 2g) in 3D, n_x + 2g in
 * 2D, x fastest; a packed low-side buffer is the neighbour's high-side ghost
 * content and vice versa.  With g = order ghost planes every zone that a
 * subdomain reconstructs sees the same stencils as in the undivided grid, so
 * the subdomains' steps together equal the undivided step bit for bit.  The
 * gate is refused on such grids (AWE_ERR_ARG at awe_create): its flags need
 * stencils beyond the ghost planes, and the two sides of an exchanged face
 * would reconstruct the zones beside it differently. */
/* Doubles in one halo buffer. */
int awe_halo_size(const awe_grid* g, size_t* count);
/* Pack the planes next to face `side` (0 = low, 1 = high) of the state that the
 * next stage reads, with their inner-dimension ghost zones filled first (at
 * the stage's boundary time).  on_device: 1 = device pointer (enqueued on the
 * grid's stream), 0 = host pointer (synchronises). */
int awe_halo_pack(awe_grid* g, int side, double* buf, int on_device);
/* Write a neighbour's packed planes into the ghost planes beyond face `side` of
 * the state that the next stage reads.  Same pointer conventions. */
int awe_halo_unpack(awe_grid* g, int side, const double* buf, int on_device);
/* Stages of one step: 1 for ADER, the Runge-Kutta stage count for SSPRK. */
int awe_stage_count(const awe_grid* g, int* stages);
/* Run stage k of the current step (k must be the next one: 0, 1, ...).
 * Stage 0 takes dt as awe_step does (dt > 0, or the device-resident dt);
 * the last stage finishes the step (t += dt, device dt = cfl / signal-speed
 * max of this subdomain's updated state).  awe_step runs all stages at once
 * and is refused (AWE_ERR_STATE) on a multi-stage grid with exchanged faces,
 * whose ghosts must be exchanged between the stages. */
int awe_stage(awe_grid* g, int k, double dt);
/* The device-resident dt (the one awe_step(g, 0, ...) uses): read or write it
 * through a host pointer (synchronises) or a device pointer (enqueued), so
 * that the subdomains of a decomposition can take the minimum of their dt
 * (= cfl / max of their signal speeds) without a host round trip. */
int awe_get_dt(awe_grid* g, double* dt, int on_device);
int awe_set_dt(awe_grid* g, const double* dt, int on_device);
/* Number of box zones (active zones and one layer around them, per
 * reconstruction: once per step for ADER, once per stage for SSPRK) whose
 * face states went to the positivity fallback (cfg.fallback) since the last
 * call; resets the count and synchronises.  Not in the paper. */
int awe_fallback_count(awe_grid* g, long long* zones);

/* ---- per-stage probes (same kernels as awe_step, for row-by-row parity) ----
 * The box is the active zones plus one layer on each side, [-1, n_d] in each
 * dimension.  Modes of a zone are ordered a fastest: for c in 0..N, for b in
 * 0..N-c, for a in 0..N-b-c (c = 0 in 2D); the basis is Legendre on the zone
 * [-1/2,1/2] with unit leading coefficient (1, xi, xi^2-1/12, xi^3-3xi/20). */
/* Spatial modes of every box zone after reconstruction of the current state:
 * host buffer [var][mode][box z][box y][box x], FP64 (promoted in FP32 form). */
int awe_probe_modes(awe_grid* g, double* W);
/* Face quadrature states of every box zone after the predictor with time step
 * dt: host buffer [dir][side][q][var][box zone], side 0 = lower face; q =
 * i_t1 + nq*(i_t2 + nq*i_time) (3D) or i_t1 + nq*i_time (2D), Gauss-Legendre
 * points with nq = 2 nodes per transverse dimension and in time at orders 3
 * and 4, nq = 1 (the face centre at mid-step) at order 2.  ADER grids only
 * (AWE_ERR_STATE otherwise), like awe_probe_fluxes. */
int awe_probe_face_states(awe_grid* g, double dt, double* FS);
/* Face-averaged Riemann fluxes of the active faces for time step dt: host buffer,
 * per direction d the block [var][faces], faces (n_x + [d==0]) x (n_y +
 * [d==1]) x (n_z + [d==2]) with x fastest, blocks concatenated over d. */
int awe_probe_fluxes(awe_grid* g, double dt, double* F);

/* ---- kernel timing (CUDA events recorded on the grid's stream) ---- */
/* Enable (1) or disable (0) per-kernel event timing of later calls; enabling
 * resets the counters. */
int awe_profile(awe_grid* g, int enable);
/* Number of kernel kinds, and per kind: name, launches and total milliseconds
 * since timing was enabled (synchronises). */
int awe_profile_count(void);
int awe_profile_read(awe_grid* g, int kind, const char** name, long* launches, double* total_ms);
/* ---- learned troubled-zone gate (not in the paper) ----
 * Features: for each direction d and for rho and E, the 2N differences
 * f(i+k+1-N) - f(i+k-N), k = 0..2N-1, divided by their largest magnitude
 * (0 for constant data), then that magnitude over |f(i)| + 1e-12, times 100,
 * squashed by x/(1+x); index (d*2+q)*(2N+1) + k; nin = dim*2*(2N+1).
 * MLP: features -> 32 ReLU -> 32 ReLU -> logit; packed float parameters
 * W1[32][nin], b1[32], W2[32][32], b2[32], w3[32], b3. */
int awe_gate_dims(int dim, int order, int* nin, size_t* nparams);
/* Copy gate parameters in (host pointer, nparams floats). */
int awe_gate_set_weights(awe_grid* g, const float* params, size_t n);
/* Features of every ghosted zone of the current state (zeros where the
 * stencil does not fit): buffer [ghosted zone][nin], ghosted zones
 * (n_x+2g) x (n_y+2g) x (n_z+2g | 1), g = order.  on_device selects the
 * pointer kind. */
int awe_gate_features(awe_grid* g, float* feat, int on_device);
/* Labels of every ghosted zone (1 troubled, 0 smooth, 255 no stencil): max
 * over directions, over rho and E, over candidates of |omega_k - lin_k| > tau
 * for the pure-direction reconstruction of the zone means. */
int awe_gate_labels(awe_grid* g, double tau, unsigned char* labels, int on_device);
/* Gate flags of every ghosted zone: logit > 0 (FP32, fixed summation order)
 * dilated over face neighbours; zones without a stencil are flagged. */
int awe_gate_flags(awe_grid* g, unsigned char* flags, int on_device);
/* Fraction counters of the last gated step: zones reconstructed with full
 * WENO and total box zones. */
int awe_gate_stats(awe_grid* g, long* flagged, long* total);

/* MLP training on the GPU with the library's own forward/backward kernels.
 * All pointers are device pointers on the current device; X [rows][nin],
 * y [rows] in {0,1}; params/m/v hold nparams floats (Adam moments, zeroed by
 * the caller at step 0).  Each step draws `batch` rows with a counter-based
 * generator from (seed, step index), computes the mean logistic loss and its
 * gradient (deterministic fixed-order reductions, no float atomics) and
 * applies Adam (beta1 0.9, beta2 0.999, eps 1e-8, lr).  step0 is the index of
 * the first step (for the bias correction and the row draws).  loss_out
 * (device, may be NULL) receives the loss of each step [steps]. */
int awe_mlp_train(int nin, float* params, float* m, float* v, const float* X, const float* y,
                  long rows, int batch, int steps, long step0, float lr, unsigned long long seed,
                  float* loss_out, void* stream);
/* Mean logistic loss (FP32) and its gradient for the first B rows (device
 * pointers; grad has nparams floats, loss one float). */
int awe_mlp_loss_grad(int nin, const float* params, const float* X, const float* y, long B,
                      float* grad, float* loss, void* stream);
/* Logits of B rows in the gate's FP32 decision order (device pointers). */
int awe_mlp_forward(int nin, const float* params, const float* X, long B, float* z, void* stream);

/* ---- time step without device allocation ----
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory when they need a time step (a runtime that plans
 * all device memory ahead and forbids allocation during a step, a component
 * under a fixed device-memory budget, a time loop that must not fail on an
 * allocation).  Same value as awe_cfl_dt, dt = cfl / max over zones of
 * max_d (|v_d| + c)/dx_d, for a state the caller holds:
 *   U   device pointer, conserved variables [var][z][y][x], active zones only
 *       (the awe_get_state layout), nvar = dim + 2, read only;
 *   n   zone counts (dim entries), dx zone sizes (dim entries), host pointers;
 *   dt  device pointer to one double (caller owned), written by the GPU;
 *   stream  cudaStream_t (NULL = default stream); the call only enqueues.
 * It allocates nothing: its scratch (one partial maximum per 4096 zones) is a
 * fixed 512 KB array inside the library, present on every GPU that loads it
 * until the process exits, so grids above 268,435,456 zones are rejected
 * (AWE_ERR_ARG, message in awe_last_error(NULL)).  The first call on each
 * device looks up that array's device address; make it before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that destroys and re-creates the device's
 * primary context) this entry point must not be called again in that
 * process.  All calls share the array: calls that overlap on the GPU race and
 * must be serialised by the caller.  dt = 0 signals a non-physical or
 * non-finite zone.  U and dt are not checked for extent (the C ABI cannot
 * see it): U must hold (dim + 2) * prod(n) doubles. */
int awe_cfl_dt_noalloc(const double* U, int dim, const int* n, const double* dx, double gamma,
                       double cfl, double* dt, void* stream);

/* ---- hardware probe ----
 * Sustained FMA throughput of this GPU in TFLOP/s (FMA = 2 flops), FP64 and
 * FP32, measured by a register-resident FMA kernel with CUDA events. */
int awe_measure_fma_peaks(double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif
#endif
