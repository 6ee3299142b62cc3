/*
 * ora.h -- plain FP64 CPU oracle for the ADER-WENO Euler zone update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library,
 * its Python binding) may include, link or call this code; only the tests,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / --impl reference legs
 * use it.  It shares no code, header, table or constant generator with the
 * CUDA path.
 *
 * The method is the three-stage scheme of the paper (Sec. II.2, Figs. 1-7):
 * WENO reconstruction of the conserved variables, an ADER predictor that
 * extends each zone's polynomial in time, and a Riemann-solver corrector whose
 * face fluxes update the zone means, followed by the CFL reduction of Fig. 7.
 * The paper names the ingredients but gives no formulas; the readings used
 * here (basis, stencils, weights, Picard predictor, Riemann solvers,
 * quadrature, BCs, the Runge-Kutta variant) are stated one by one in the
 * comments of ora.c.
 *
 * Layout of every state array: conserved variables, structure of arrays,
 * [var][z][y][x], x fastest.  "Ghosted" arrays carry g = order ghost zones on
 * each side of every active dimension (none along z in 2D).
 */
#ifndef ORA_H
#define ORA_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_BC_PERIODIC = 0, ORA_BC_OUTFLOW = 1, ORA_BC_REFLECT = 2,
       ORA_BC_INFLOW = 3, ORA_BC_DMR_BOTTOM = 4, ORA_BC_DMR_TOP = 5 };

typedef struct {
  int dim;              /* 2 or 3 */
  int n[3];             /* active zones per dimension (n[2] = 1 in 2D) */
  int order;            /* 2, 3 or 4; polynomial degree N = order - 1 (order 2 uses
                           the paper's MC limiter instead of WENO) */
  int picard;           /* number of Picard sweeps K of the predictor */
  double lo[3], hi[3];  /* domain box */
  double gamma;         /* ratio of specific heats */
  double eps;           /* WENO epsilon (absolute) */
  double lin[4];        /* linear weights of the r candidate stencils */
  int bc[6];            /* xlo, xhi, ylo, yhi, zlo, zhi */
  double inflow[6][5];  /* fixed conserved state per face (inflow / DMR post-shock) */
  double pre[5];        /* DMR pre-shock conserved state (top boundary) */
  int fallback;         /* 1: positivity fallback of the face states; 2: that and the
                           a posteriori first-order update of non-physical zones
                           (see ora.c) */
  int riemann;          /* ORA_RS_*: Riemann solver of the corrector (HLLC by default) */
} ora_cfg;

/* ---- small building blocks (exported for the pins) ---- */
void ora_gauss_legendre(int n, double* x, double* w);          /* on [-1/2, 1/2] */
double ora_basis(int a, double xi);                             /* scaled Legendre P_a */
int ora_num_modes(int dim, int N);                              /* spatial modes, total degree <= N */
int ora_num_st_modes(int dim, int N);                           /* space-time modes */
void ora_mode_list(int dim, int N, int* abc);                   /* [nmodes][3] */
void ora_candidate(int N, int k, const double* u, double* coef);/* stencil k of 1D recon */
double ora_beta(int N, const double* coef);                     /* smoothness of a candidate */
void ora_weno1d(int N, const double* u, double eps, const double* lin,
                int linear_only, double* coef, double* omega);
double ora_mc_slope(double a, double b, double cfac);           /* order-2 limiter, Fig. 3 */
enum { ORA_RS_HLLC = 0, ORA_RS_HLL = 1, ORA_RS_HLLEM = 2, ORA_RS_RUSANOV = 3 };
void ora_hllc(int dim, double gamma, int dir, const double* UL, const double* UR, double* F);
void ora_hll(int dim, double gamma, int dir, const double* UL, const double* UR, double* F);
void ora_hllem(int dim, double gamma, int dir, const double* UL, const double* UR, double* F);
void ora_rusanov(int dim, double gamma, int dir, const double* UL, const double* UR, double* F);
void ora_riemann(int kind, int dim, double gamma, int dir, const double* UL, const double* UR,
                 double* F);
void ora_phys_flux(int dim, double gamma, int dir, const double* U, double* F);

/* ---- whole-grid operations ---- */
size_t ora_ghosted_size(const ora_cfg* c);                      /* zones per variable */
int ora_fill_ghosts(const ora_cfg* c, double* Ug, double t);
/* Spatial modes of every zone of the box [-1, n_d] (all active dims).
 * W layout [var][mode][box zone]; flags (ghosted zone count, may be NULL):
 * 0 -> linear weights, else full WENO. */
int ora_reconstruct(const ora_cfg* c, const double* Ug, const unsigned char* flags, double* W);
/* Predictor of one zone: w[var][mode] -> space-time coefficients st[var][st-mode]. */
void ora_predict_zone(const ora_cfg* c, const double* w, double dt, double* st);
/* Face quadrature states of every box zone: FS[dir][side][q][var][box zone];
 * returns the number of box zones sent to the positivity fallback. */
int ora_face_states(const ora_cfg* c, const double* Ug, const unsigned char* flags,
                    double dt, double* FS);
/* One full step on a ghost-filled state. Uout: active zones [var][z][y][x].
 * smax: max over updated zones of max_d (|v_d| + c)/dx_d (dt_next = cfl/smax).
 * Returns 0, or -4 if the updated state is non-physical / non-finite. */
int ora_step(const ora_cfg* c, const double* Ug, double dt, const unsigned char* flags,
             double* Uout, double* smax);
/* Face-averaged fluxes of active faces: F[dir][var][face], face grid (n_d+1) along dir. */
int ora_fluxes(const ora_cfg* c, const double* Ug, const unsigned char* flags, double dt, double* F);
double ora_signal_max(const ora_cfg* c, const double* Ug);
/* Runge-Kutta variant (Table IV's comparison scheme; see ora.c): Shu-Osher
 * coefficients of the SSP scheme with 2, 3 or 5 stages ([stages+1][stages],
 * row i = stage i), L(U) of a ghost-filled state on the active zones, and
 * one whole step from an active state at time t. */
int ora_rk_coefficients(int stages, double* alpha, double* beta);
int ora_rk_rhs(const ora_cfg* c, const double* Ug, const unsigned char* flags, double* L);
int ora_rk_step(const ora_cfg* c, const double* U, double t, double dt, int stages, int nh,
                const float* gate_params, double* Uout, double* smax);

/* ---- exact Riemann solver (ideal gas) sampled at x/t = s ---- */
int ora_exact_riemann(double gamma, double rl, double ul, double pl,
                      double rr, double ur, double pr, double s,
                      double* r, double* u, double* p, double* pstar, double* ustar);

/* ---- troubled-zone gate: labels, features, MLP ---- */
int ora_gate_num_features(int dim, int order);
/* Labels over ghosted zones (1 = troubled), 255 where the stencil does not fit. */
int ora_weno_labels(const ora_cfg* c, const double* Ug, double tau, unsigned char* labels);
/* Features over ghosted zones [zone][feature] as float; zones without a full stencil get 0. */
int ora_gate_features(const ora_cfg* c, const double* Ug, float* feat);
size_t ora_mlp_num_params(int nin, int nh);
/* FP64 forward: logits z[b] for B rows of x[b][nin]; params in float (packed). */
void ora_mlp_forward_f64(int nin, int nh, const float* params, const float* x, int B, double* z);
/* FP64 mean-BCE loss and its gradient w.r.t. the packed parameters. */
double ora_mlp_loss_grad_f64(int nin, int nh, const float* params, const float* x,
                             const float* y, int B, double* grad);
/* FP32 forward in a fixed summation order (the gate decision precision). */
void ora_mlp_forward_f32(int nin, int nh, const float* params, const float* x, int B, float* z);
/* Gate flags over ghosted zones: logit > 0, dilated over face neighbours;
 * zones without features are flagged. */
int ora_gate_flags(const ora_cfg* c, const double* Ug, int nh, const float* params,
                   unsigned char* flags);

#ifdef __cplusplus
}
#endif
#endif
