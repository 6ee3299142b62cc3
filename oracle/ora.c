/*
 * ora.c -- plain FP64 CPU oracle of the ADER-WENO Euler zone update.
 *
 * TEST INFRASTRUCTURE ONLY (see ora.h): not part of the product path, and it
 * shares no code with the CUDA library.  Written for reading, not speed:
 * every operator is evaluated from its definition with naive loops over
 * quadrature nodes and modes (no sum factorisation, no fusion).  Compile with
 * -ffp-contract=off so that no operation is fused behind the reader's back.
 *
 * Structure follows the paper's time step (Sec. II.2, Fig. 1): ghost zones
 * (Boundary_Conditions), reconstruction (Limiter, Fig. 3, here WENO at order
 * 3/4), predictor (Fig. 4), face fluxes from a Riemann solver (Fig. 5), the
 * flux difference (Fig. 6) and the update with the CFL reduction (Fig. 7).
 *
 * Readings the paper does not fix (its refs [9], [10], [12], [22], [40] are
 * not part of the text) are stated where they are used; parity is pinned by
 * the oracle tests (tests/test_oracle_*.py), not by this file.
 */
#include "ora.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXN 3          /* highest polynomial degree (order 4) */
#define MAXM 20         /* spatial modes, 3D, N = 3 */
#define MAXST 35        /* space-time modes, 3D, N = 3 */
#define MAXV 5          /* conserved variables in 3D */

/* ------------------------------------------------------------------------ */
/* Quadrature and basis                                                      */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes/weights on [-1/2, 1/2] (weights sum to 1), ascending
 * nodes, by Newton iteration on the Legendre recurrence. */
void ora_gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = -0.5 * z;
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Reading: modal basis in space is Legendre on the zone [-1/2, 1/2] scaled to
 * unit leading coefficient, so that mode 1 is the undivided slope: the paper's
 * O2 face value is mean +/- 1/2 slope (Fig. 5). */
double ora_basis(int a, double x) {
  switch (a) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return x * x - 1.0 / 12.0;
    case 3: return x * x * x - (3.0 / 20.0) * x;
  }
  return 0.0;
}
static double basis_deriv(int a, double x) {
  switch (a) {
    case 1: return 1.0;
    case 2: return 2.0 * x;
    case 3: return 3.0 * x * x - 3.0 / 20.0;
  }
  return 0.0;
}
/* monomial coefficients of P_a (m[j] multiplies x^j) */
static void basis_monomials(int a, double* m) {
  for (int j = 0; j <= MAXN; ++j) m[j] = 0.0;
  switch (a) {
    case 0: m[0] = 1.0; break;
    case 1: m[1] = 1.0; break;
    case 2: m[0] = -1.0 / 12.0; m[2] = 1.0; break;
    case 3: m[1] = -3.0 / 20.0; m[3] = 1.0; break;
  }
}
/* Time basis: shifted Legendre on [0, 1]; only the represented polynomial
 * matters, not this choice. */
static double tbasis(int e, double t) {
  switch (e) {
    case 0: return 1.0;
    case 1: return 2.0 * t - 1.0;
    case 2: return 6.0 * t * t - 6.0 * t + 1.0;
    case 3: return 20.0 * t * t * t - 30.0 * t * t + 12.0 * t - 1.0;
  }
  return 0.0;
}
/* integral from 0 to t of tbasis(e) */
static double tbasis_int(int e, double t) {
  switch (e) {
    case 0: return t;
    case 1: return t * t - t;
    case 2: return 2.0 * t * t * t - 3.0 * t * t + t;
    case 3: return 5.0 * t * t * t * t - 10.0 * t * t * t + 6.0 * t * t - t;
  }
  return 0.0;
}

static int binom(int n, int k) {
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
int ora_num_modes(int dim, int N) { return binom(N + dim, dim); }
int ora_num_st_modes(int dim, int N) { return binom(N + dim + 1, dim + 1); }

/* Spatial modes (a, b, c) of total degree <= N, a fastest:
 * for c = 0..N, b = 0..N-c, a = 0..N-b-c.  In 2D c = 0. */
void ora_mode_list(int dim, int N, int* abc) {
  int m = 0;
  int cmax = dim == 3 ? N : 0;
  for (int c = 0; c <= cmax; ++c)
    for (int b = 0; b <= N - c; ++b)
      for (int a = 0; a <= N - b - c; ++a) {
        abc[3 * m + 0] = a;
        abc[3 * m + 1] = b;
        abc[3 * m + 2] = c;
        ++m;
      }
}
/* Space-time modes (a, b, c, e), time index outermost, same inner order. */
static int st_mode_list(int dim, int N, int* abce) {
  int m = 0;
  int cmax = dim == 3 ? N : 0;
  for (int e = 0; e <= N; ++e)
    for (int c = 0; c <= (cmax < N - e ? cmax : N - e); ++c)
      for (int b = 0; b <= N - e - c; ++b)
        for (int a = 0; a <= N - e - b - c; ++a) {
          abce[4 * m + 0] = a;
          abce[4 * m + 1] = b;
          abce[4 * m + 2] = c;
          abce[4 * m + 3] = e;
          ++m;
        }
  return m;
}
static int st_index(int dim, int N, const int* abce_list, int nst, int a, int b, int c, int e) {
  (void)dim; (void)N;
  for (int m = 0; m < nst; ++m)
    if (abce_list[4 * m] == a && abce_list[4 * m + 1] == b && abce_list[4 * m + 2] == c &&
        abce_list[4 * m + 3] == e)
      return m;
  return -1;
}

/* ------------------------------------------------------------------------ */
/* 1D WENO reconstruction (per conserved component)                          */
/* ------------------------------------------------------------------------ */
/* Reading (the paper names finite-volume WENO of the conserved variables,
 * Sec. I.1, without formulas): r = N+1 candidate stencils, each r zones wide
 * ({k-N .. k} for k = 0..N), each fitted with a full degree-N polynomial whose
 * zone averages match the data; nonlinear weights
 * omega_k ~ lin_k / (eps + beta_k)^2 with beta_k the sum over derivative
 * orders l = 1..N of the integral over the zone of (d^l p / dxi^l)^2.  The
 * zone mean is kept as the zone average. */

/* average of P_a over the zone at offset s (by Gauss quadrature, exact);
 * tabulated once when the library is loaded, for |s| <= MAXN */
static double zone_avg_table[MAXN + 1][2 * MAXN + 1];
__attribute__((constructor)) static void ora_tables_init(void) {
  double x[MAXN + 2], w[MAXN + 2];
  ora_gauss_legendre(MAXN + 1, x, w);
  for (int a = 0; a <= MAXN; ++a)
    for (int s = -MAXN; s <= MAXN; ++s) {
      double acc = 0.0;
      for (int q = 0; q <= MAXN; ++q) acc += w[q] * ora_basis(a, (double)s + x[q]);
      zone_avg_table[a][s + MAXN] = acc;
    }
}
static double basis_zone_average(int a, int s) { return zone_avg_table[a][s + MAXN]; }

/* Candidate k: u holds the 2N+1 zone averages at offsets -N..N (u[N] is the
 * zone itself).  Solves for the modal coefficients coef[0..N-1] (modes 1..N). */
void ora_candidate(int N, int k, const double* u, double* coef) {
  double A[MAXN][MAXN + 1];
  int row = 0;
  for (int s = k - N; s <= k; ++s) {
    if (s == 0) continue;
    for (int a = 1; a <= N; ++a) A[row][a - 1] = basis_zone_average(a, s);
    A[row][N] = u[N + s] - u[N];
    ++row;
  }
  /* Gaussian elimination with partial pivoting */
  for (int col = 0; col < N; ++col) {
    int piv = col;
    for (int r = col + 1; r < N; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (piv != col)
      for (int j = 0; j <= N; ++j) {
        double t = A[col][j];
        A[col][j] = A[piv][j];
        A[piv][j] = t;
      }
    for (int r = col + 1; r < N; ++r) {
      double f = A[r][col] / A[col][col];
      for (int j = col; j <= N; ++j) A[r][j] -= f * A[col][j];
    }
  }
  for (int r = N - 1; r >= 0; --r) {
    double acc = A[r][N];
    for (int j = r + 1; j < N; ++j) acc -= A[r][j] * coef[j];
    coef[r] = acc / A[r][r];
  }
}

/* beta = sum_{l=1..N} int_{-1/2}^{1/2} (d^l p/dxi^l)^2 dxi, p = sum_a coef[a-1] P_a,
 * evaluated from the monomial form by Gauss quadrature (exact). */
double ora_beta(int N, const double* coef) {
  double m[MAXN + 1] = {0}, pm[MAXN + 1];
  for (int a = 1; a <= N; ++a) {
    basis_monomials(a, pm);
    for (int j = 0; j <= MAXN; ++j) m[j] += coef[a - 1] * pm[j];
  }
  double x[MAXN + 2], w[MAXN + 2];
  ora_gauss_legendre(N + 1, x, w);
  double beta = 0.0;
  for (int l = 1; l <= N; ++l) {
    for (int q = 0; q <= N; ++q) {
      double d = 0.0;
      for (int j = l; j <= N; ++j) {
        double f = 1.0;
        for (int t = 0; t < l; ++t) f *= (double)(j - t);
        d += m[j] * f * pow(x[q], (double)(j - l));
      }
      beta += w[q] * d * d;
    }
  }
  return beta;
}

void ora_weno1d(int N, const double* u, double eps, const double* lin, int linear_only,
                double* coef, double* omega) {
  double cand[MAXN + 1][MAXN];
  double alpha[MAXN + 1], asum = 0.0;
  for (int k = 0; k <= N; ++k) {
    ora_candidate(N, k, u, cand[k]);
    if (linear_only) {
      alpha[k] = lin[k];
    } else {
      double b = ora_beta(N, cand[k]);
      alpha[k] = lin[k] / ((eps + b) * (eps + b));
    }
    asum += alpha[k];
  }
  for (int a = 0; a < N; ++a) coef[a] = 0.0;
  for (int k = 0; k <= N; ++k) {
    double om = alpha[k] / asum;
    if (omega) omega[k] = om;
    for (int a = 0; a < N; ++a) coef[a] += om * cand[k][a];
  }
}

/* Order 2: the paper's own limiter (Fig. 3).  The slope of a zone from its
 * two one-sided differences a = u(i+1)-u(i), b = u(i)-u(i-1) is
 * min(|a+b|/2, cfac|a|, cfac|b|) when a and b have the same sign and 0
 * otherwise (the listing's SIGN(0.5,a) + SIGN(0.5,b) factor, with SIGN
 * taking the sign of its second argument and +0.5 at zero); the compression
 * factor is 2.0 for the density and 1.5 for the other variables. */
double ora_mc_slope(double a, double b, double cfac) {
  double m = fmin(0.5 * fabs(a + b), fmin(cfac * fabs(a), cfac * fabs(b)));
  double sa = a >= 0.0 ? 0.5 : -0.5, sb = b >= 0.0 ? 0.5 : -0.5;
  return m * (sa + sb);
}

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  int dim, N, g, nv;
  int n[3], G[3];     /* active and ghosted extents (G[2] = 1 in 2D) */
  size_t ntot;
  double dx[3];
} geom;

static void make_geom(const ora_cfg* c, geom* q) {
  q->dim = c->dim;
  q->N = c->order - 1;
  q->g = c->order;
  q->nv = c->dim + 2;
  for (int d = 0; d < 3; ++d) {
    q->n[d] = (d < c->dim) ? c->n[d] : 1;
    q->G[d] = (d < c->dim) ? c->n[d] + 2 * q->g : 1;
    q->dx[d] = (d < c->dim) ? (c->hi[d] - c->lo[d]) / c->n[d] : 1.0;
  }
  q->ntot = (size_t)q->G[0] * q->G[1] * q->G[2];
}
static size_t gidx(const geom* q, int i, int j, int k) {
  return ((size_t)k * q->G[1] + j) * q->G[0] + i;
}
static int zone_physical(const geom* q, double gamma, const double* U);
size_t ora_ghosted_size(const ora_cfg* c) {
  geom q;
  make_geom(c, &q);
  return q.ntot;
}

/* ------------------------------------------------------------------------ */
/* Boundary conditions (ghost zones)                                         */
/* ------------------------------------------------------------------------ */
/* The paper fills ghost zones in Boundary_Conditions before the limiter
 * (Fig. 1).  Reading: BCs are applied dimension after dimension (x, then y,
 * then z), so a corner ghost is the z-image of a y-image of an x-image.
 * Periodic: wrap.  Outflow: copy of the nearest active zone.  Reflect: mirror
 * image with the normal momentum negated.  Inflow: fixed state.  DMR bottom:
 * post-shock inflow state for x < 1/6, reflecting wall beyond.  DMR top: the
 * exact moving-shock state at the ghost zone's x, evaluated at the start of the
 * step: post-shock if x < 1/6 + (1 + 20 t)/sqrt(3), else pre-shock. */
static void ghost_value(const ora_cfg* c, const geom* q, const double* Ug, int idx[3], double t,
                        double* out) {
  for (int d = q->dim - 1; d >= 0; --d) {
    int lo = q->g, hi = q->g + q->n[d];
    if (idx[d] >= lo && idx[d] < hi) continue;
    int side = idx[d] < lo ? 0 : 1;
    int bc = c->bc[2 * d + side];
    int m[3] = {idx[0], idx[1], idx[2]};
    double xc = c->lo[0] + (idx[0] - q->g + 0.5) * q->dx[0];
    switch (bc) {
      case ORA_BC_PERIODIC: {
        int r = (idx[d] - lo) % q->n[d];
        if (r < 0) r += q->n[d];
        m[d] = lo + r;
        ghost_value(c, q, Ug, m, t, out);
        return;
      }
      case ORA_BC_OUTFLOW:
        m[d] = side ? hi - 1 : lo;
        ghost_value(c, q, Ug, m, t, out);
        return;
      case ORA_BC_DMR_BOTTOM:
        if (xc < 1.0 / 6.0) {
          for (int v = 0; v < q->nv; ++v) out[v] = c->inflow[2 * d + side][v];
          return;
        }
        /* fall through: reflecting wall */
      case ORA_BC_REFLECT:
        m[d] = side ? 2 * hi - 1 - idx[d] : 2 * lo - 1 - idx[d];
        ghost_value(c, q, Ug, m, t, out);
        out[1 + d] = -out[1 + d];
        return;
      case ORA_BC_INFLOW:
        for (int v = 0; v < q->nv; ++v) out[v] = c->inflow[2 * d + side][v];
        return;
      case ORA_BC_DMR_TOP: {
        double xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / sqrt(3.0);
        const double* s = (xc < xs) ? c->inflow[2 * d + side] : c->pre;
        for (int v = 0; v < q->nv; ++v) out[v] = s[v];
        return;
      }
      default:
        for (int v = 0; v < q->nv; ++v) out[v] = NAN;
        return;
    }
  }
  for (int v = 0; v < q->nv; ++v) out[v] = Ug[v * q->ntot + gidx(q, idx[0], idx[1], idx[2])];
}

int ora_fill_ghosts(const ora_cfg* c, double* Ug, double t) {
  geom q;
  make_geom(c, &q);
  for (int k = 0; k < q.G[2]; ++k)
    for (int j = 0; j < q.G[1]; ++j)
      for (int i = 0; i < q.G[0]; ++i) {
        int idx[3] = {i, j, k};
        int inside = 1;
        for (int d = 0; d < q.dim; ++d)
          if (idx[d] < q.g || idx[d] >= q.g + q.n[d]) inside = 0;
        if (inside) continue;
        double v[MAXV];
        ghost_value(c, &q, Ug, idx, t, v);
        for (int s = 0; s < q.nv; ++s) Ug[s * q.ntot + gidx(&q, i, j, k)] = v[s];
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Multidimensional reconstruction                                           */
/* ------------------------------------------------------------------------ */
/* Reading: the pure modes along each axis come from the 1D recon of the zone
 * averages along that axis; a mixed mode comes from the 1D recon, along the
 * later axis, of the field of an already built mode (u_xy = y-slope of the u_x
 * field, u_xyy = y-curvature of u_x, u_xxy = y-slope of u_xx, likewise with z,
 * and u_xyz = z-slope of the u_xy field).  Every 1D recon at a zone uses that
 * zone's gate flag (0: linear weights). */

/* recon along dimension d of field f at every zone whose stencil fits and whose
 * inputs are finite; out[a] (a = 0..N-1) receives coefficient of P_{a+1} */
static void recon_field(const ora_cfg* c, const geom* q, const double* f, int d,
                        const unsigned char* flags, double** out, int nout, double cfac) {
  const int N = q->N;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < q->G[2]; ++k)
    for (int j = 0; j < q->G[1]; ++j)
      for (int i = 0; i < q->G[0]; ++i) {
        int idx[3] = {i, j, k};
        size_t z = gidx(q, i, j, k);
        for (int a = 0; a < nout; ++a) out[a][z] = NAN;
        if (idx[d] < N || idx[d] > q->G[d] - 1 - N) continue;
        double u[2 * MAXN + 1];
        int ok = 1;
        for (int s = -N; s <= N; ++s) {
          int m[3] = {i, j, k};
          m[d] += s;
          u[N + s] = f[gidx(q, m[0], m[1], m[2])];
          if (!isfinite(u[N + s])) ok = 0;
        }
        if (!ok) continue;
        double coef[MAXN], om[MAXN + 1];
        if (N == 1) {
          coef[0] = ora_mc_slope(u[2] - u[1], u[1] - u[0], cfac);
        } else {
          int lin_only = flags ? (flags[z] == 0) : 0;
          ora_weno1d(N, u, c->eps, c->lin, lin_only, coef, om);
        }
        for (int a = 0; a < nout; ++a) out[a][z] = coef[a];
      }
}

int ora_reconstruct(const ora_cfg* c, const double* Ug, const unsigned char* flags, double* W) {
  geom q;
  make_geom(c, &q);
  const int N = q.N, dim = q.dim;
  const int ns = ora_num_modes(dim, N);
  int modes[MAXM * 3];
  ora_mode_list(dim, N, modes);
  int B[3];
  for (int d = 0; d < 3; ++d) B[d] = d < dim ? q.n[d] + 2 : 1;
  const size_t nbox = (size_t)B[0] * B[1] * B[2];

  /* field storage: fld[a][b][c] holds the mode (a,b,c) field; (0,0,0) = averages */
  double* fld[MAXN + 1][MAXN + 1][MAXN + 1];
  memset(fld, 0, sizeof(fld));
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N - a; ++b)
      for (int cc = 0; cc <= N - a - b; ++cc) {
        if (dim == 2 && cc > 0) continue;
        fld[a][b][cc] = (double*)malloc(q.ntot * sizeof(double));
      }

  for (int v = 0; v < q.nv; ++v) {
    memcpy(fld[0][0][0], Ug + (size_t)v * q.ntot, q.ntot * sizeof(double));
    double* outs[MAXN];
    /* x family: pure x modes from the averages */
    for (int a = 1; a <= N; ++a) outs[a - 1] = fld[a][0][0];
    const double cfac = v == 0 ? 2.0 : 1.5; /* order-2 limiter compression factor */
    recon_field(c, &q, fld[0][0][0], 0, flags, outs, N, cfac);
    /* y family: recon along y of every (a,0,0) field, keep b = 1..N-a */
    for (int a = 0; a < N; ++a) {
      for (int b = 1; b <= N - a; ++b) outs[b - 1] = fld[a][b][0];
      recon_field(c, &q, fld[a][0][0], 1, flags, outs, N - a, cfac);
    }
    /* z family: recon along z of every (a,b,0) field, keep c = 1..N-a-b */
    if (dim == 3)
      for (int b = 0; b < N; ++b)
        for (int a = 0; a < N - b; ++a) {
          for (int cc = 1; cc <= N - a - b; ++cc) outs[cc - 1] = fld[a][b][cc];
          recon_field(c, &q, fld[a][b][0], 2, flags, outs, N - a - b, cfac);
        }
    for (int kb = 0; kb < B[2]; ++kb)
      for (int jb = 0; jb < B[1]; ++jb)
        for (int ib = 0; ib < B[0]; ++ib) {
          int i = ib - 1 + q.g, j = dim >= 2 ? jb - 1 + q.g : jb, k = dim == 3 ? kb - 1 + q.g : 0;
          size_t z = gidx(&q, i, j, k);
          size_t bz = ((size_t)kb * B[1] + jb) * B[0] + ib;
          for (int m = 0; m < ns; ++m) {
            const double* f = fld[modes[3 * m]][modes[3 * m + 1]][modes[3 * m + 2]];
            W[((size_t)v * ns + m) * nbox + bz] = f[z];
          }
        }
  }
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N; ++b)
      for (int cc = 0; cc <= N; ++cc) free(fld[a][b][cc]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Physical flux and HLLC                                                    */
/* ------------------------------------------------------------------------ */
/* Euler flux along direction dir of the conserved state U (ideal gas,
 * p = (gamma-1)(E - rho|v|^2/2)). */
void ora_phys_flux(int dim, double gamma, int dir, const double* U, double* F) {
  const int nv = dim + 2;
  double rho = U[0];
  double v[3] = {0, 0, 0}, kin = 0.0;
  for (int d = 0; d < dim; ++d) {
    v[d] = U[1 + d] / rho;
    kin += 0.5 * rho * v[d] * v[d];
  }
  double E = U[nv - 1];
  double p = (gamma - 1.0) * (E - kin);
  double un = v[dir];
  F[0] = rho * un;
  for (int d = 0; d < dim; ++d) F[1 + d] = rho * un * v[d] + (d == dir ? p : 0.0);
  F[nv - 1] = (E + p) * un;
}

/* HLLC (Toro, Spruce and Speares; named in Sec. I.1).  Reading: Davis-Einfeldt
 * wave speeds with Roe averages, S_L = min(u_L - c_L, u~ - c~),
 * S_R = max(u_R + c_R, u~ + c~); the middle wave speed S* from the usual
 * pressure balance; at S* = 0 the left star state is used. */
void ora_hllc(int dim, double gamma, int dir, const double* UL, const double* UR, double* F) {
  const int nv = dim + 2;
  double rl = UL[0], rr = UR[0];
  double vl[3] = {0, 0, 0}, vr[3] = {0, 0, 0};
  double kl = 0.0, kr = 0.0;
  for (int d = 0; d < dim; ++d) {
    vl[d] = UL[1 + d] / rl;
    vr[d] = UR[1 + d] / rr;
    kl += 0.5 * rl * vl[d] * vl[d];
    kr += 0.5 * rr * vr[d] * vr[d];
  }
  double El = UL[nv - 1], Er = UR[nv - 1];
  double pl = (gamma - 1.0) * (El - kl), pr = (gamma - 1.0) * (Er - kr);
  double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
  double ul = vl[dir], ur = vr[dir];
  double sl = sqrt(rl), sr = sqrt(rr);
  double vt[3] = {0, 0, 0}, vt2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    vt[d] = (sl * vl[d] + sr * vr[d]) / (sl + sr);
    vt2 += vt[d] * vt[d];
  }
  double Hl = (El + pl) / rl, Hr = (Er + pr) / rr;
  double Ht = (sl * Hl + sr * Hr) / (sl + sr);
  double ct = sqrt((gamma - 1.0) * (Ht - 0.5 * vt2));
  double SL = fmin(ul - cl, vt[dir] - ct);
  double SR = fmax(ur + cr, vt[dir] + ct);
  double Ss = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) /
              (rl * (SL - ul) - rr * (SR - ur));
  double FL[MAXV], FR[MAXV];
  ora_phys_flux(dim, gamma, dir, UL, FL);
  ora_phys_flux(dim, gamma, dir, UR, FR);
  if (0.0 <= SL) {
    for (int s = 0; s < nv; ++s) F[s] = FL[s];
  } else if (0.0 <= Ss) {
    double f = rl * (SL - ul) / (SL - Ss);
    double Us[MAXV];
    Us[0] = f;
    for (int d = 0; d < dim; ++d) Us[1 + d] = f * (d == dir ? Ss : vl[d]);
    Us[nv - 1] = f * (El / rl + (Ss - ul) * (Ss + pl / (rl * (SL - ul))));
    for (int s = 0; s < nv; ++s) F[s] = FL[s] + SL * (Us[s] - UL[s]);
  } else if (0.0 < SR) {
    double f = rr * (SR - ur) / (SR - Ss);
    double Us[MAXV];
    Us[0] = f;
    for (int d = 0; d < dim; ++d) Us[1 + d] = f * (d == dir ? Ss : vr[d]);
    Us[nv - 1] = f * (Er / rr + (Ss - ur) * (Ss + pr / (rr * (SR - ur))));
    for (int s = 0; s < nv; ++s) F[s] = FR[s] + SR * (Us[s] - UR[s]);
  } else {
    for (int s = 0; s < nv; ++s) F[s] = FR[s];
  }
}

/* The other Riemann solvers the paper names beside HLLC (Sec. I.1): HLL,
 * HLLEM and Rusanov.  Readings (the paper gives no formulas):
 *  - HLL (Harten, Lax and van Leer): the single intermediate state between the
 *    Davis-Einfeldt speeds S_L, S_R of ora_hllc; F = F_L if 0 <= S_L, F_R if
 *    S_R <= 0, else (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
 *  - HLLEM (Einfeldt; in the anti-diffusive form of Dumbser and Balsara):
 *    HLL with the linearly degenerate waves (the contact and the dim-1 shear
 *    waves, all moving with the Roe velocity u~) restored.  Their Roe
 *    strengths are a_c = drho - dp/c~^2 along r_c = (1, v~, |v~|^2/2) and
 *    a_t = rho~ dv_t along r_t = (0, e_t, v~_t); inside the fan the HLL jump
 *    term S_L S_R dU becomes S_L S_R (dU - delta sum_k a_k r_k) with
 *    delta = 1 - min(u~,0)/S_L - max(u~,0)/S_R, which makes isolated
 *    contacts and shear waves exact for any speeds bracketing u~.
 *  - Rusanov (local Lax-Friedrichs): F = (F_L + F_R)/2 - S (U_R - U_L)/2 with
 *    S = max(|u_L| + c_L, |u_R| + c_R), the normal velocity u. */
typedef struct {
  double rl, rr, vl[3], vr[3], pl, pr, cl, cr, El, Er;
  double rt, vt[3], vt2, ct, SL, SR;
} ora_rs_states;

static void rs_states(int dim, double gamma, int dir, const double* UL, const double* UR,
                      ora_rs_states* w) {
  const int nv = dim + 2;
  w->rl = UL[0];
  w->rr = UR[0];
  double kl = 0.0, kr = 0.0;
  for (int d = 0; d < 3; ++d) w->vl[d] = w->vr[d] = w->vt[d] = 0.0;
  for (int d = 0; d < dim; ++d) {
    w->vl[d] = UL[1 + d] / w->rl;
    w->vr[d] = UR[1 + d] / w->rr;
    kl += 0.5 * w->rl * w->vl[d] * w->vl[d];
    kr += 0.5 * w->rr * w->vr[d] * w->vr[d];
  }
  w->El = UL[nv - 1];
  w->Er = UR[nv - 1];
  w->pl = (gamma - 1.0) * (w->El - kl);
  w->pr = (gamma - 1.0) * (w->Er - kr);
  w->cl = sqrt(gamma * w->pl / w->rl);
  w->cr = sqrt(gamma * w->pr / w->rr);
  double sl = sqrt(w->rl), sr = sqrt(w->rr);
  w->rt = sl * sr;
  w->vt2 = 0.0;
  for (int d = 0; d < dim; ++d) {
    w->vt[d] = (sl * w->vl[d] + sr * w->vr[d]) / (sl + sr);
    w->vt2 += w->vt[d] * w->vt[d];
  }
  double Hl = (w->El + w->pl) / w->rl, Hr = (w->Er + w->pr) / w->rr;
  double Ht = (sl * Hl + sr * Hr) / (sl + sr);
  w->ct = sqrt((gamma - 1.0) * (Ht - 0.5 * w->vt2));
  w->SL = fmin(w->vl[dir] - w->cl, w->vt[dir] - w->ct);
  w->SR = fmax(w->vr[dir] + w->cr, w->vt[dir] + w->ct);
}

/* HLL and HLLEM share everything but the restored waves (hllem = 0 or 1). */
static void hll_family(int dim, double gamma, int dir, const double* UL, const double* UR,
                       int hllem, double* F) {
  const int nv = dim + 2;
  ora_rs_states w;
  rs_states(dim, gamma, dir, UL, UR, &w);
  double FL[MAXV], FR[MAXV];
  ora_phys_flux(dim, gamma, dir, UL, FL);
  ora_phys_flux(dim, gamma, dir, UR, FR);
  if (0.0 <= w.SL) {
    for (int s = 0; s < nv; ++s) F[s] = FL[s];
    return;
  }
  if (w.SR <= 0.0) {
    for (int s = 0; s < nv; ++s) F[s] = FR[s];
    return;
  }
  double jump[MAXV];
  for (int s = 0; s < nv; ++s) jump[s] = UR[s] - UL[s];
  if (hllem) {
    double ut = w.vt[dir];
    double delta = 1.0 - fmin(ut, 0.0) / w.SL - fmax(ut, 0.0) / w.SR;
    double ac = (w.rr - w.rl) - (w.pr - w.pl) / (w.ct * w.ct);
    double rwave[MAXV];
    /* contact */
    rwave[0] = 1.0;
    for (int d = 0; d < dim; ++d) rwave[1 + d] = w.vt[d];
    rwave[nv - 1] = 0.5 * w.vt2;
    for (int s = 0; s < nv; ++s) jump[s] -= delta * ac * rwave[s];
    /* shear waves */
    for (int t = 0; t < dim; ++t) {
      if (t == dir) continue;
      double at = w.rt * (w.vr[t] - w.vl[t]);
      for (int s = 0; s < nv; ++s) rwave[s] = 0.0;
      rwave[1 + t] = 1.0;
      rwave[nv - 1] = w.vt[t];
      for (int s = 0; s < nv; ++s) jump[s] -= delta * at * rwave[s];
    }
  }
  for (int s = 0; s < nv; ++s)
    F[s] = (w.SR * FL[s] - w.SL * FR[s] + w.SL * w.SR * jump[s]) / (w.SR - w.SL);
}

void ora_hll(int dim, double gamma, int dir, const double* UL, const double* UR, double* F) {
  hll_family(dim, gamma, dir, UL, UR, 0, F);
}

void ora_hllem(int dim, double gamma, int dir, const double* UL, const double* UR, double* F) {
  hll_family(dim, gamma, dir, UL, UR, 1, F);
}

void ora_rusanov(int dim, double gamma, int dir, const double* UL, const double* UR, double* F) {
  const int nv = dim + 2;
  ora_rs_states w;
  rs_states(dim, gamma, dir, UL, UR, &w);
  double FL[MAXV], FR[MAXV];
  ora_phys_flux(dim, gamma, dir, UL, FL);
  ora_phys_flux(dim, gamma, dir, UR, FR);
  double S = fmax(fabs(w.vl[dir]) + w.cl, fabs(w.vr[dir]) + w.cr);
  for (int s = 0; s < nv; ++s) F[s] = 0.5 * (FL[s] + FR[s]) - 0.5 * S * (UR[s] - UL[s]);
}

void ora_riemann(int kind, int dim, double gamma, int dir, const double* UL, const double* UR,
                 double* F) {
  switch (kind) {
    case ORA_RS_HLL: ora_hll(dim, gamma, dir, UL, UR, F); break;
    case ORA_RS_HLLEM: ora_hllem(dim, gamma, dir, UL, UR, F); break;
    case ORA_RS_RUSANOV: ora_rusanov(dim, gamma, dir, UL, UR, F); break;
    default: ora_hllc(dim, gamma, dir, UL, UR, F); break;
  }
}

/* ------------------------------------------------------------------------ */
/* ADER predictor                                                            */
/* ------------------------------------------------------------------------ */
/* The paper's Predictor_Ptwise (Fig. 4) builds, zone by zone, the time
 * dependence of the reconstructed polynomial from the PDE itself.  Reading
 * (local space-time Picard form of the ADER predictor):
 *   q^0(xi, tau) = w(xi),
 *   q^{k+1} = w - int_0^tau sum_d (dt/dx_d) d/dxi_d Pi_N[F_d(q^k)] dtau',
 * k = 0..K-1, where Pi_N is the L2 projection onto space-time polynomials of
 * total degree <= N over [-1/2,1/2]^d x [0,1], its inner products taken with the
 * tensor Gauss-Legendre rule of N+1 nodes per dimension (space and time).
 * The derivative lowers and the time integral restores the degree, so q^{k+1}
 * stays of total degree <= N. */
void ora_predict_zone(const ora_cfg* c, const double* w, double dt, double* st) {
  geom q;
  make_geom(c, &q);
  const int dim = q.dim, N = q.N, nv = q.nv;
  const int ns = ora_num_modes(dim, N);
  int smodes[MAXM * 3], stm[MAXST * 4];
  ora_mode_list(dim, N, smodes);
  const int nst = st_mode_list(dim, N, stm);
  const int nn = N + 1;
  double xg[MAXN + 1], wg[MAXN + 1], tg[MAXN + 1];
  ora_gauss_legendre(nn, xg, wg);
  for (int i = 0; i < nn; ++i) tg[i] = xg[i] + 0.5;

  /* norms and the derivative / time-integral tables, all by quadrature */
  double nP[MAXN + 1], nL[MAXN + 1];
  for (int a = 0; a <= N; ++a) {
    nP[a] = 0.0;
    nL[a] = 0.0;
    for (int i = 0; i < nn; ++i) {
      nP[a] += wg[i] * ora_basis(a, xg[i]) * ora_basis(a, xg[i]);
      nL[a] += wg[i] * tbasis(a, tg[i]) * tbasis(a, tg[i]);
    }
  }
  double D[MAXN + 1][MAXN + 1], I[MAXN + 1][MAXN + 1];
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N; ++b) {
      double sd = 0.0, si = 0.0;
      for (int i = 0; i < nn; ++i) {
        sd += wg[i] * basis_deriv(a, xg[i]) * ora_basis(b, xg[i]);
        si += wg[i] * tbasis_int(a, tg[i]) * tbasis(b, tg[i]);
      }
      D[a][b] = sd / nP[b]; /* coefficient of P_b in dP_a/dxi */
      I[a][b] = si / nL[b]; /* coefficient of L_b in int_0^tau L_a */
      if (fabs(D[a][b]) < 1e-13) D[a][b] = 0.0;
      if (fabs(I[a][b]) < 1e-13) I[a][b] = 0.0;
    }

  double cur[MAXV][MAXST], nxt[MAXV][MAXST];
  double proj[3][MAXV][MAXST];
  for (int v = 0; v < nv; ++v)
    for (int m = 0; m < nst; ++m) cur[v][m] = 0.0;
  for (int v = 0; v < nv; ++v)
    for (int m = 0; m < ns; ++m) {
      int idx = st_index(dim, N, stm, nst, smodes[3 * m], smodes[3 * m + 1], smodes[3 * m + 2], 0);
      cur[v][idx] = w[v * ns + m];
    }

  const int nz_nodes = dim == 3 ? nn : 1;
  for (int sweep = 0; sweep < c->picard; ++sweep) {
    memset(proj, 0, sizeof(proj));
    for (int it = 0; it < nn; ++it)
      for (int i2 = 0; i2 < nz_nodes; ++i2)
        for (int i1 = 0; i1 < nn; ++i1)
          for (int i0 = 0; i0 < nn; ++i0) {
            double wt = wg[i0] * wg[i1] * wg[it] * (dim == 3 ? wg[i2] : 1.0);
            double phi[MAXST];
            for (int m = 0; m < nst; ++m) {
              phi[m] = ora_basis(stm[4 * m], xg[i0]) * ora_basis(stm[4 * m + 1], xg[i1]) *
                       (dim == 3 ? ora_basis(stm[4 * m + 2], xg[i2]) : 1.0) *
                       tbasis(stm[4 * m + 3], tg[it]);
            }
            double qn[MAXV];
            for (int v = 0; v < nv; ++v) {
              qn[v] = 0.0;
              for (int m = 0; m < nst; ++m) qn[v] += cur[v][m] * phi[m];
            }
            for (int d = 0; d < dim; ++d) {
              double F[MAXV];
              ora_phys_flux(dim, c->gamma, d, qn, F);
              for (int v = 0; v < nv; ++v)
                for (int m = 0; m < nst; ++m) proj[d][v][m] += wt * F[v] * phi[m];
            }
          }
    for (int d = 0; d < dim; ++d)
      for (int v = 0; v < nv; ++v)
        for (int m = 0; m < nst; ++m) {
          double nrm = nP[stm[4 * m]] * nP[stm[4 * m + 1]] * (dim == 3 ? nP[stm[4 * m + 2]] : 1.0) *
                       nL[stm[4 * m + 3]];
          proj[d][v][m] /= nrm;
        }
    /* q^{k+1} = w - sum_d (dt/dx_d) int_0^tau d/dxi_d Pi_N F_d */
    for (int v = 0; v < nv; ++v)
      for (int m = 0; m < nst; ++m) nxt[v][m] = 0.0;
    for (int v = 0; v < nv; ++v)
      for (int m = 0; m < ns; ++m) {
        int idx = st_index(dim, N, stm, nst, smodes[3 * m], smodes[3 * m + 1], smodes[3 * m + 2], 0);
        nxt[v][idx] = w[v * ns + m];
      }
    for (int d = 0; d < dim; ++d) {
      double lam = dt / q.dx[d];
      for (int v = 0; v < nv; ++v)
        for (int m = 0; m < nst; ++m) {
          int al[3] = {stm[4 * m], stm[4 * m + 1], stm[4 * m + 2]};
          int e = stm[4 * m + 3];
          if (al[d] < 1) continue;
          for (int ap = 0; ap < al[d]; ++ap) {
            if (D[al[d]][ap] == 0.0) continue;
            for (int ep = 0; ep <= e + 1 && ep <= N; ++ep) {
              if (I[e][ep] == 0.0) continue;
              int bl[3] = {al[0], al[1], al[2]};
              bl[d] = ap;
              int t = st_index(dim, N, stm, nst, bl[0], bl[1], bl[2], ep);
              if (t < 0) continue; /* cannot happen: degree drops by >= 1, rises by <= 1 */
              nxt[v][t] -= lam * proj[d][v][m] * D[al[d]][ap] * I[e][ep];
            }
          }
        }
    }
    memcpy(cur, nxt, sizeof(cur));
  }
  for (int v = 0; v < nv; ++v)
    for (int m = 0; m < nst; ++m) st[v * nst + m] = cur[v][m];
}

static double st_eval(int dim, int nst, const int* stm, const double* coef, const double* xi,
                      double tau) {
  double acc = 0.0;
  for (int m = 0; m < nst; ++m) {
    double phi = ora_basis(stm[4 * m], xi[0]) * ora_basis(stm[4 * m + 1], xi[1]) *
                 (dim == 3 ? ora_basis(stm[4 * m + 2], xi[2]) : 1.0) * tbasis(stm[4 * m + 3], tau);
    acc += coef[m] * phi;
  }
  return acc;
}

/* ------------------------------------------------------------------------ */
/* Face quadrature states                                                    */
/* ------------------------------------------------------------------------ */
/* Reading: the corrector averages the Riemann flux over the face and the time
 * step with a tensor Gauss-Legendre rule of nq = ceil(order/2) nodes per
 * transverse dimension and in time: 2 at orders 3 and 4, and at order 2 the
 * paper's single mid-face, mid-step point (Fig. 5).  Point index
 * q = i_t1 + nq*(i_t2 + nq*i_time) in 3D (t1 < t2 the transverse dimensions),
 * q = i_t1 + nq*i_time in 2D. */
#define NQMAX 2
int ora_face_states(const ora_cfg* c, const double* Ug, const unsigned char* flags, double dt,
                    double* FS) {
  geom q;
  make_geom(c, &q);
  const int dim = q.dim, N = q.N, nv = q.nv;
  const int ns = ora_num_modes(dim, N), nst = ora_num_st_modes(dim, N);
  int stm[MAXST * 4];
  st_mode_list(dim, N, stm);
  int B[3];
  for (int d = 0; d < 3; ++d) B[d] = d < dim ? q.n[d] + 2 : 1;
  const size_t nbox = (size_t)B[0] * B[1] * B[2];
  const int NQ = (c->order + 1) / 2;
  const int nfq = dim == 3 ? NQ * NQ * NQ : NQ * NQ;
  double* W = (double*)malloc(sizeof(double) * nv * ns * nbox);
  ora_reconstruct(c, Ug, flags, W);
  double xq[NQMAX], wq[NQMAX];
  ora_gauss_legendre(NQ, xq, wq);
  long nfallback = 0;
#pragma omp parallel for schedule(static) reduction(+ : nfallback)
  for (long bz = 0; bz < (long)nbox; ++bz) {
    double w[MAXV * MAXM], st[MAXV * MAXST];
    for (int v = 0; v < nv; ++v)
      for (int m = 0; m < ns; ++m) w[v * ns + m] = W[((size_t)v * ns + m) * nbox + bz];
    ora_predict_zone(c, w, dt, st);
    int bad = 0;
    for (int d = 0; d < dim; ++d) {
      int t1 = -1, t2 = -1;
      for (int e = 0; e < dim; ++e)
        if (e != d) {
          if (t1 < 0) t1 = e; else t2 = e;
        }
      for (int side = 0; side < 2; ++side)
        for (int p = 0; p < nfq; ++p) {
          int i1 = p % NQ, i2 = dim == 3 ? (p / NQ) % NQ : 0, it = dim == 3 ? p / (NQ * NQ) : p / NQ;
          double xi[3] = {0, 0, 0};
          xi[d] = side ? 0.5 : -0.5;
          xi[t1] = xq[i1];
          if (t2 >= 0) xi[t2] = xq[i2];
          double tau = xq[it] + 0.5;
          double U[MAXV];
          for (int v = 0; v < nv; ++v) {
            U[v] = st_eval(dim, nst, stm, st + v * nst, xi, tau);
            FS[((((size_t)d * 2 + side) * nfq + p) * nv + v) * nbox + bz] = U[v];
          }
          if (!zone_physical(&q, c->gamma, U)) bad = 1;
        }
    }
    /* Positivity fallback (not in the paper; opt-in): a zone with a face
     * state of non-positive density or pressure (or a non-finite one) falls
     * back to first order: all its face states become the zone mean. */
    if (c->fallback && bad) {
      nfallback += 1;
      for (int d = 0; d < dim; ++d)
        for (int side = 0; side < 2; ++side)
          for (int p = 0; p < nfq; ++p)
            for (int v = 0; v < nv; ++v)
              FS[((((size_t)d * 2 + side) * nfq + p) * nv + v) * nbox + bz] = w[v * ns + 0];
    }
  }
  free(W);
  return (int)nfallback;
}

/* Face-averaged Riemann fluxes of the active faces (Make_Flux_X/Y/Z, Fig. 5):
 * F[dir][var][face], faces along dir indexed 0..n_dir (face f is the lower face
 * of active zone f), x fastest. */
int ora_fluxes(const ora_cfg* c, const double* Ug, const unsigned char* flags, double dt, double* F) {
  geom q;
  make_geom(c, &q);
  const int dim = q.dim, nv = q.nv;
  int B[3];
  for (int d = 0; d < 3; ++d) B[d] = d < dim ? q.n[d] + 2 : 1;
  const size_t nbox = (size_t)B[0] * B[1] * B[2];
  const int NQ = (c->order + 1) / 2;
  const int nfq = dim == 3 ? NQ * NQ * NQ : NQ * NQ;
  double* FS = (double*)malloc(sizeof(double) * dim * 2 * nfq * nv * nbox);
  ora_face_states(c, Ug, flags, dt, FS);
  double xq[NQMAX], wq[NQMAX];
  ora_gauss_legendre(NQ, xq, wq);
  size_t off = 0;
  for (int d = 0; d < dim; ++d) {
    int E[3] = {q.n[0], q.n[1], q.n[2]};
    E[d] += 1;
    size_t nf = (size_t)E[0] * E[1] * E[2];
#pragma omp parallel for schedule(static)
    for (long f = 0; f < (long)nf; ++f) {
      int fi[3] = {(int)(f % E[0]), (int)((f / E[0]) % E[1]), (int)(f / ((size_t)E[0] * E[1]))};
      /* box coordinates of the zones left (lower) and right (upper) of the face */
      int lb[3], rb[3];
      for (int e = 0; e < 3; ++e) {
        int base = e < dim ? fi[e] + 1 : 0;
        lb[e] = base;
        rb[e] = base;
      }
      lb[d] -= 1;
      size_t lz = ((size_t)lb[2] * B[1] + lb[1]) * B[0] + lb[0];
      size_t rz = ((size_t)rb[2] * B[1] + rb[1]) * B[0] + rb[0];
      double acc[MAXV] = {0, 0, 0, 0, 0};
      for (int p = 0; p < nfq; ++p) {
        int i1 = p % NQ, i2 = dim == 3 ? (p / NQ) % NQ : 0, it = dim == 3 ? p / (NQ * NQ) : p / NQ;
        double wt = wq[i1] * wq[it] * (dim == 3 ? wq[i2] : 1.0);
        double UL[MAXV], UR[MAXV], Fp[MAXV];
        for (int v = 0; v < nv; ++v) {
          UL[v] = FS[((((size_t)d * 2 + 1) * nfq + p) * nv + v) * nbox + lz];
          UR[v] = FS[((((size_t)d * 2 + 0) * nfq + p) * nv + v) * nbox + rz];
        }
        ora_riemann(c->riemann, dim, c->gamma, d, UL, UR, Fp);
        for (int v = 0; v < nv; ++v) acc[v] += wt * Fp[v];
      }
      for (int v = 0; v < nv; ++v) F[off + (size_t)v * nf + f] = acc[v];
    }
    off += (size_t)nv * nf;
  }
  free(FS);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Update and CFL reduction                                                  */
/* ------------------------------------------------------------------------ */
/* Signal speed of one zone: max_d (|v_d| + c)/dx_d.  The paper reduces the
 * per-zone time step with a MIN (Fig. 7); reading: dt_next = cfl / max over
 * zones of this signal speed (identical to the MIN of cfl*dx/(|v|+c) up to
 * rounding). */
static double zone_signal(const geom* q, double gamma, const double* U) {
  double rho = U[0], kin = 0.0, v[3] = {0, 0, 0};
  for (int d = 0; d < q->dim; ++d) {
    v[d] = U[1 + d] / rho;
    kin += 0.5 * rho * v[d] * v[d];
  }
  double p = (gamma - 1.0) * (U[q->nv - 1] - kin);
  double cs = sqrt(gamma * p / rho);
  double s = 0.0;
  for (int d = 0; d < q->dim; ++d) {
    double sd = (fabs(v[d]) + cs) / q->dx[d];
    if (sd > s) s = sd;
  }
  return s;
}
static int zone_physical(const geom* q, double gamma, const double* U) {
  for (int v = 0; v < q->nv; ++v)
    if (!isfinite(U[v])) return 0;
  double rho = U[0], kin = 0.0;
  if (!(rho > 0.0)) return 0;
  for (int d = 0; d < q->dim; ++d) kin += 0.5 * U[1 + d] * U[1 + d] / rho;
  double p = (gamma - 1.0) * (U[q->nv - 1] - kin);
  return p > 0.0;
}

double ora_signal_max(const ora_cfg* c, const double* Ug) {
  geom q;
  make_geom(c, &q);
  double smax = 0.0;
  for (int k = 0; k < q.n[2]; ++k)
    for (int j = 0; j < q.n[1]; ++j)
      for (int i = 0; i < q.n[0]; ++i) {
        int gi = i + q.g, gj = q.dim >= 2 ? j + q.g : j, gk = q.dim == 3 ? k + q.g : 0;
        double U[MAXV];
        for (int v = 0; v < q.nv; ++v) U[v] = Ug[v * q.ntot + gidx(&q, gi, gj, gk)];
        double s = zone_signal(&q, c->gamma, U);
        if (s > smax) smax = s;
      }
  return smax;
}

/* A posteriori fallback (not in the paper; fallback = 2).  After the update,
 * a zone whose new mean is not physical is flagged; every flagged zone and
 * every zone sharing a face with one is updated again from the old state,
 * with the flux of each face next to a flagged zone replaced by the Riemann
 * flux between the two old zone means (first order), the high-order flux on
 * every other face.  Both zones of a face use the same flux, so the update
 * stays conservative; a fully first-order zone stays physical under the
 * positivity condition of the first-order scheme (its CFL sum below 1/2).
 * Flags accumulate over ORA_FB_PASSES passes (a zone that a first-order
 * neighbour makes non-physical is flagged in the next pass).  Across a
 * periodic face the neighbour is the periodic image; other boundary faces
 * have no neighbour to flag. */
#define ORA_FB_PASSES 4
static int fb_neighbour(const geom* q, int idx[3], int d, int s, const ora_cfg* c, size_t* out) {
  int m[3] = {idx[0], idx[1], idx[2]};
  m[d] += s;
  if (m[d] < 0 || m[d] >= q->n[d]) {
    if (c->bc[2 * d + (s > 0)] != 0) return 0; /* not periodic: no neighbour */
    m[d] = (m[d] + q->n[d]) % q->n[d];
  }
  *out = ((size_t)m[2] * q->n[1] + m[1]) * q->n[0] + m[0];
  return 1;
}

static void a_posteriori_fallback(const ora_cfg* c, const geom* q, const double* Ug, double dt, const double* F,
                                  const size_t* offs, const size_t* nfs, double* Uout) {
  const int dim = q->dim, nv = q->nv;
  const size_t nact = (size_t)q->n[0] * q->n[1] * q->n[2];
  unsigned char* fl = (unsigned char*)calloc(nact, 1);
  double* Unew = (double*)malloc(sizeof(double) * nv * nact);
  for (int pass = 0; pass < ORA_FB_PASSES; ++pass) {
    for (size_t z = 0; z < nact; ++z) {
      double U[MAXV];
      for (int v = 0; v < nv; ++v) U[v] = Uout[(size_t)v * nact + z];
      if (!zone_physical(q, c->gamma, U)) fl[z] = 1;
    }
    memcpy(Unew, Uout, sizeof(double) * nv * nact);
    for (size_t z = 0; z < nact; ++z) {
      int idx[3] = {(int)(z % q->n[0]), (int)((z / q->n[0]) % q->n[1]), (int)(z / ((size_t)q->n[0] * q->n[1]))};
      /* flags of the zone and of its neighbours below (s = -1) and above (s = +1) in each direction */
      int near = fl[z], nfl[3][2] = {{0, 0}, {0, 0}, {0, 0}};
      for (int d = 0; d < dim; ++d)
        for (int si = 0; si < 2; ++si) {
          size_t w;
          if (fb_neighbour(q, idx, d, si ? 1 : -1, c, &w) && fl[w]) {
            nfl[d][si] = 1;
            near = 1;
          }
        }
      if (!near) continue;
      int gi = idx[0] + q->g, gj = dim >= 2 ? idx[1] + q->g : idx[1], gk = dim == 3 ? idx[2] + q->g : 0;
      double U0[MAXV];
      for (int v = 0; v < nv; ++v) U0[v] = Ug[v * q->ntot + gidx(q, gi, gj, gk)];
      double acc[MAXV] = {0, 0, 0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        int E[3] = {q->n[0], q->n[1], q->n[2]};
        E[d] += 1;
        double Ffo[2][MAXV];  /* faces below (0) and above (1) */
        for (int si = 0; si < 2; ++si) {
          int fi[3] = {idx[0], idx[1], idx[2]};
          fi[d] += si;
          size_t f = ((size_t)fi[2] * E[1] + fi[1]) * E[0] + fi[0];
          if (fl[z] || nfl[d][si]) {
            int m[3] = {gi, gj, gk};
            m[d] += si ? 1 : -1;
            double Un[MAXV], *UL = si ? U0 : Un, *UR = si ? Un : U0;
            for (int v = 0; v < nv; ++v) Un[v] = Ug[v * q->ntot + gidx(q, m[0], m[1], m[2])];
            ora_riemann(c->riemann, dim, c->gamma, d, UL, UR, Ffo[si]);
          } else {
            for (int v = 0; v < nv; ++v) Ffo[si][v] = F[offs[d] + (size_t)v * nfs[d] + f];
          }
        }
        for (int v = 0; v < nv; ++v) acc[v] += (dt / q->dx[d]) * (Ffo[1][v] - Ffo[0][v]);
      }
      for (int v = 0; v < nv; ++v) Unew[(size_t)v * nact + z] = U0[v] - acc[v];
    }
    memcpy(Uout, Unew, sizeof(double) * nv * nact);
  }
  free(Unew);
  free(fl);
}

/* One step (Make_dU_dt and Update_U_Timestep, Figs. 6-7):
 * U+ = U - dt * sum_d (F_{d,i+1/2} - F_{d,i-1/2}) / dx_d on the active zones. */
int ora_step(const ora_cfg* c, const double* Ug, double dt, const unsigned char* flags, double* Uout,
             double* smax) {
  geom q;
  make_geom(c, &q);
  const int dim = q.dim, nv = q.nv;
  size_t nfl = 0, offs[3];
  size_t nfs[3];
  for (int d = 0; d < dim; ++d) {
    int E[3] = {q.n[0], q.n[1], q.n[2]};
    E[d] += 1;
    nfs[d] = (size_t)E[0] * E[1] * E[2];
    offs[d] = nfl;
    nfl += (size_t)nv * nfs[d];
  }
  double* F = (double*)malloc(sizeof(double) * nfl);
  ora_fluxes(c, Ug, flags, dt, F);
  const size_t nact = (size_t)q.n[0] * q.n[1] * q.n[2];
  int bad = 0;
  double sm = 0.0;
  for (size_t z = 0; z < nact; ++z) {
    int i = (int)(z % q.n[0]), j = (int)((z / q.n[0]) % q.n[1]), k = (int)(z / ((size_t)q.n[0] * q.n[1]));
    int gi = i + q.g, gj = dim >= 2 ? j + q.g : j, gk = dim == 3 ? k + q.g : 0;
    double U[MAXV];
    for (int v = 0; v < nv; ++v) {
      double acc = 0.0;
      for (int d = 0; d < dim; ++d) {
        int E[3] = {q.n[0], q.n[1], q.n[2]};
        E[d] += 1;
        int lo[3] = {i, j, k}, hi[3] = {i, j, k};
        hi[d] += 1;
        size_t fl = ((size_t)lo[2] * E[1] + lo[1]) * E[0] + lo[0];
        size_t fh = ((size_t)hi[2] * E[1] + hi[1]) * E[0] + hi[0];
        acc += (dt / q.dx[d]) * (F[offs[d] + (size_t)v * nfs[d] + fh] - F[offs[d] + (size_t)v * nfs[d] + fl]);
      }
      U[v] = Ug[v * q.ntot + gidx(&q, gi, gj, gk)] - acc;
      Uout[(size_t)v * nact + z] = U[v];
    }
    if (!zone_physical(&q, c->gamma, U)) bad = 1;
    double s = zone_signal(&q, c->gamma, U);
    if (s > sm) sm = s;
  }
  if (c->fallback == 2) {
    a_posteriori_fallback(c, &q, Ug, dt, F, offs, nfs, Uout);
    bad = 0;
    sm = 0.0;
    for (size_t z = 0; z < nact; ++z) {
      double U[MAXV];
      for (int v = 0; v < nv; ++v) U[v] = Uout[(size_t)v * nact + z];
      if (!zone_physical(&q, c->gamma, U)) bad = 1;
      double s = zone_signal(&q, c->gamma, U);
      if (s > sm) sm = s;
    }
  }
  free(F);
  if (smax) *smax = sm;
  return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* Runge-Kutta variant (method of lines; Table IV's comparison scheme)        */
/* ------------------------------------------------------------------------ */
/* The paper compares ADER with Runge-Kutta time stepping of the same WENO
 * reconstruction and Riemann fluxes (Sec. IV, Table IV): two stages at second
 * order, three at third and five at fourth.  Reading: strong-stability-
 * preserving schemes in Shu-Osher form,
 *   U(i) = sum_{k<i} [ alpha_ik U(k) + beta_ik dt L(U(k)) ],  U(0) = U^n,
 * with L(U) = -sum_d (F_{d,i+1/2} - F_{d,i-1/2}) / dx_d, the face fluxes the
 * Gauss average over the face only (no time points: nq = ceil(order/2) per
 * transverse dimension) of the Riemann solver between the reconstructed
 * polynomials of the two zones.  Schemes: SSP(2,2) (Heun), SSP(3,3)
 * (Shu and Osher) and the five-stage fourth-order SSP(5,4) of Spiteri and
 * Ruuth.  The boundary values of stage k are those at time t + c_k dt, with
 * the stage abscissae c_i = sum_k (alpha_ik c_k + beta_ik). */
#define RK_MAXS 5
static int rk_table(int stages, double alpha[RK_MAXS + 1][RK_MAXS], double beta[RK_MAXS + 1][RK_MAXS]) {
  for (int i = 0; i <= RK_MAXS; ++i)
    for (int k = 0; k < RK_MAXS; ++k) alpha[i][k] = beta[i][k] = 0.0;
  if (stages == 2) {
    alpha[1][0] = 1.0; beta[1][0] = 1.0;
    alpha[2][0] = 0.5; alpha[2][1] = 0.5; beta[2][1] = 0.5;
    return 0;
  }
  if (stages == 3) {
    alpha[1][0] = 1.0; beta[1][0] = 1.0;
    alpha[2][0] = 0.75; alpha[2][1] = 0.25; beta[2][1] = 0.25;
    alpha[3][0] = 1.0 / 3.0; alpha[3][2] = 2.0 / 3.0; beta[3][2] = 2.0 / 3.0;
    return 0;
  }
  if (stages == 5) {
    alpha[1][0] = 1.0;               beta[1][0] = 0.391752226571890;
    alpha[2][0] = 0.444370493651235; alpha[2][1] = 0.555629506348765; beta[2][1] = 0.368410593050371;
    alpha[3][0] = 0.620101851488403; alpha[3][2] = 0.379898148511597; beta[3][2] = 0.251891774271694;
    alpha[4][0] = 0.178079954393132; alpha[4][3] = 0.821920045606868; beta[4][3] = 0.544974750228521;
    alpha[5][2] = 0.517231671970585; alpha[5][3] = 0.096059710526147; beta[5][3] = 0.063692468666290;
    alpha[5][4] = 0.386708617503269; beta[5][4] = 0.226007483236906;
    return 0;
  }
  return -1;
}

int ora_rk_coefficients(int stages, double* alpha, double* beta) {
  double a[RK_MAXS + 1][RK_MAXS], b[RK_MAXS + 1][RK_MAXS];
  if (rk_table(stages, a, b)) return -1;
  for (int i = 0; i <= stages; ++i)
    for (int k = 0; k < stages; ++k) {
      alpha[i * stages + k] = a[i][k];
      beta[i * stages + k] = b[i][k];
    }
  return 0;
}

/* L(U) on the active zones, [var][active zone], from a ghost-filled state. */
int ora_rk_rhs(const ora_cfg* c, const double* Ug, const unsigned char* flags, double* L) {
  geom q;
  make_geom(c, &q);
  const int dim = q.dim, N = q.N, nv = q.nv;
  const int ns = ora_num_modes(dim, N);
  int abc[MAXM * 3];
  ora_mode_list(dim, N, abc);
  int B[3];
  for (int d = 0; d < 3; ++d) B[d] = d < dim ? q.n[d] + 2 : 1;
  const size_t nbox = (size_t)B[0] * B[1] * B[2];
  const int NQ = (c->order + 1) / 2;
  const int np = dim == 3 ? NQ * NQ : NQ;   /* points per face, space only */
  double* W = (double*)malloc(sizeof(double) * nv * ns * nbox);
  double* FS = (double*)malloc(sizeof(double) * dim * 2 * np * nv * nbox);
  ora_reconstruct(c, Ug, flags, W);
  double xq[NQMAX], wq[NQMAX];
  ora_gauss_legendre(NQ, xq, wq);
  /* face states: the reconstructed polynomial at the face points */
#pragma omp parallel for schedule(static)
  for (long bz = 0; bz < (long)nbox; ++bz) {
    int bad = 0;
    for (int d = 0; d < dim; ++d) {
      int t1 = -1, t2 = -1;
      for (int e = 0; e < dim; ++e)
        if (e != d) {
          if (t1 < 0) t1 = e; else t2 = e;
        }
      for (int side = 0; side < 2; ++side)
        for (int p = 0; p < np; ++p) {
          double xi[3] = {0, 0, 0};
          xi[d] = side ? 0.5 : -0.5;
          xi[t1] = xq[p % NQ];
          if (t2 >= 0) xi[t2] = xq[p / NQ];
          double U[MAXV];
          for (int v = 0; v < nv; ++v) {
            double acc = 0.0;
            for (int m = 0; m < ns; ++m) {
              double b = 1.0;
              for (int e = 0; e < dim; ++e) b *= ora_basis(abc[m * 3 + e], xi[e]);
              acc += W[((size_t)v * ns + m) * nbox + bz] * b;
            }
            U[v] = acc;
            FS[((((size_t)d * 2 + side) * np + p) * nv + v) * nbox + bz] = acc;
          }
          if (!zone_physical(&q, c->gamma, U)) bad = 1;
        }
    }
    if (c->fallback && bad) {
      for (int d = 0; d < dim; ++d)
        for (int side = 0; side < 2; ++side)
          for (int p = 0; p < np; ++p)
            for (int v = 0; v < nv; ++v)
              FS[((((size_t)d * 2 + side) * np + p) * nv + v) * nbox + bz] = W[((size_t)v * ns + 0) * nbox + bz];
    }
  }
  const size_t nact = (size_t)q.n[0] * q.n[1] * q.n[2];
  for (size_t z = 0; z < nact * nv; ++z) L[z] = 0.0;
  for (int d = 0; d < dim; ++d) {
    int E[3] = {q.n[0], q.n[1], q.n[2]};
    E[d] += 1;
    size_t nf = (size_t)E[0] * E[1] * E[2];
    double* F = (double*)malloc(sizeof(double) * nv * nf);
#pragma omp parallel for schedule(static)
    for (long f = 0; f < (long)nf; ++f) {
      int fi[3] = {(int)(f % E[0]), (int)((f / E[0]) % E[1]), (int)(f / ((size_t)E[0] * E[1]))};
      int lb[3], rb[3];
      for (int e = 0; e < 3; ++e) lb[e] = rb[e] = e < dim ? fi[e] + 1 : 0;
      lb[d] -= 1;
      size_t lz = ((size_t)lb[2] * B[1] + lb[1]) * B[0] + lb[0];
      size_t rz = ((size_t)rb[2] * B[1] + rb[1]) * B[0] + rb[0];
      double acc[MAXV] = {0, 0, 0, 0, 0};
      for (int p = 0; p < np; ++p) {
        double wt = wq[p % NQ] * (dim == 3 ? wq[p / NQ] : 1.0);
        double UL[MAXV], UR[MAXV], Fp[MAXV];
        for (int v = 0; v < nv; ++v) {
          UL[v] = FS[((((size_t)d * 2 + 1) * np + p) * nv + v) * nbox + lz];
          UR[v] = FS[((((size_t)d * 2 + 0) * np + p) * nv + v) * nbox + rz];
        }
        ora_riemann(c->riemann, dim, c->gamma, d, UL, UR, Fp);
        for (int v = 0; v < nv; ++v) acc[v] += wt * Fp[v];
      }
      for (int v = 0; v < nv; ++v) F[(size_t)v * nf + f] = acc[v];
    }
    for (size_t z = 0; z < nact; ++z) {
      int i = (int)(z % q.n[0]), j = (int)((z / q.n[0]) % q.n[1]), k = (int)(z / ((size_t)q.n[0] * q.n[1]));
      int lo[3] = {i, j, k}, hi[3] = {i, j, k};
      hi[d] += 1;
      size_t fl = ((size_t)lo[2] * E[1] + lo[1]) * E[0] + lo[0];
      size_t fh = ((size_t)hi[2] * E[1] + hi[1]) * E[0] + hi[0];
      for (int v = 0; v < nv; ++v) L[(size_t)v * nact + z] -= (F[(size_t)v * nf + fh] - F[(size_t)v * nf + fl]) / q.dx[d];
    }
    free(F);
  }
  free(W);
  free(FS);
  return 0;
}

/* One Runge-Kutta step from the active state U at time t (ghost zones are
 * filled by the boundary conditions at each stage's time); gate_params, if
 * not NULL, are the MLP weights (nh hidden units) from which each stage
 * computes its troubled-zone flags.  Returns -4 if a stage state or the
 * result is non-physical, -1 for an unknown stage count. */
int ora_rk_step(const ora_cfg* c, const double* U, double t, double dt, int stages, int nh,
                const float* gate_params, double* Uout, double* smax) {
  double alpha[RK_MAXS + 1][RK_MAXS], beta[RK_MAXS + 1][RK_MAXS];
  if (rk_table(stages, alpha, beta)) return -1;
  geom q;
  make_geom(c, &q);
  const int nv = q.nv, dim = q.dim;
  const size_t nact = (size_t)q.n[0] * q.n[1] * q.n[2];
  double* Us[RK_MAXS + 1];
  double* Ls[RK_MAXS];
  double cst[RK_MAXS + 1];
  for (int i = 0; i <= stages; ++i) Us[i] = (double*)malloc(sizeof(double) * nv * nact);
  for (int i = 0; i < stages; ++i) Ls[i] = (double*)malloc(sizeof(double) * nv * nact);
  double* Ug = (double*)malloc(sizeof(double) * nv * q.ntot);
  unsigned char* flags = gate_params ? (unsigned char*)malloc(q.ntot) : NULL;
  memcpy(Us[0], U, sizeof(double) * nv * nact);
  cst[0] = 0.0;
  int bad = 0;
  for (int i = 1; i <= stages; ++i) {
    /* L of the previous stage */
    const int k = i - 1;
    for (size_t z = 0; z < q.ntot * nv; ++z) Ug[z] = 0.0;
    for (size_t z = 0; z < nact; ++z) {
      int a = (int)(z % q.n[0]), b = (int)((z / q.n[0]) % q.n[1]), cc = (int)(z / ((size_t)q.n[0] * q.n[1]));
      size_t gz = gidx(&q, a + q.g, b + q.g, dim == 3 ? cc + q.g : 0);
      for (int v = 0; v < nv; ++v) Ug[(size_t)v * q.ntot + gz] = Us[k][(size_t)v * nact + z];
    }
    ora_fill_ghosts(c, Ug, t + cst[k] * dt);
    if (flags) ora_gate_flags(c, Ug, nh, gate_params, flags);
    ora_rk_rhs(c, Ug, flags, Ls[k]);
    /* stage i */
    cst[i] = 0.0;
    for (int kk = 0; kk < i; ++kk) cst[i] += alpha[i][kk] * cst[kk] + beta[i][kk];
    for (size_t z = 0; z < nact; ++z) {
      double Uz[MAXV];
      for (int v = 0; v < nv; ++v) {
        double acc = 0.0;
        for (int kk = 0; kk < i; ++kk)
          acc += alpha[i][kk] * Us[kk][(size_t)v * nact + z] + beta[i][kk] * dt * Ls[kk][(size_t)v * nact + z];
        Us[i][(size_t)v * nact + z] = acc;
        Uz[v] = acc;
      }
      if (!zone_physical(&q, c->gamma, Uz)) bad = 1;
    }
  }
  double sm = 0.0;
  for (size_t z = 0; z < nact; ++z) {
    double Uz[MAXV];
    for (int v = 0; v < nv; ++v) Uz[v] = Us[stages][(size_t)v * nact + z];
    double sg = zone_signal(&q, c->gamma, Uz);
    if (sg > sm) sm = sg;
  }
  memcpy(Uout, Us[stages], sizeof(double) * nv * nact);
  if (smax) *smax = sm;
  for (int i = 0; i <= stages; ++i) free(Us[i]);
  for (int i = 0; i < stages; ++i) free(Ls[i]);
  free(Ug);
  free(flags);
  return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* Exact Riemann solver (ideal gas), from the wave curves of the Euler       */
/* equations: shock branch from Rankine-Hugoniot, rarefaction branch from the */
/* isentropic Riemann invariant; p* by Newton's method on the pressure        */
/* function f_L(p) + f_R(p) + u_R - u_L = 0.                                  */
/* ------------------------------------------------------------------------ */
static void wave_curve(double gamma, double p, double rk, double pk, double ck, double* f, double* df) {
  if (p > pk) {
    double A = 2.0 / ((gamma + 1.0) * rk), Bk = (gamma - 1.0) / (gamma + 1.0) * pk;
    double s = sqrt(A / (p + Bk));
    *f = (p - pk) * s;
    *df = s * (1.0 - 0.5 * (p - pk) / (p + Bk));
  } else {
    double e = (gamma - 1.0) / (2.0 * gamma);
    *f = 2.0 * ck / (gamma - 1.0) * (pow(p / pk, e) - 1.0);
    *df = 1.0 / (rk * ck) * pow(p / pk, -(gamma + 1.0) / (2.0 * gamma));
  }
}

int ora_exact_riemann(double gamma, double rl, double ul, double pl, double rr, double ur, double pr,
                      double s, double* r, double* u, double* p, double* pstar, double* ustar) {
  double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
  if (2.0 * (cl + cr) / (gamma - 1.0) <= ur - ul) return -1; /* vacuum: not handled */
  double ps = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
  if (ps < 1e-8) ps = 1e-8;
  for (int it = 0; it < 200; ++it) {
    double fl, dfl, fr, dfr;
    wave_curve(gamma, ps, rl, pl, cl, &fl, &dfl);
    wave_curve(gamma, ps, rr, pr, cr, &fr, &dfr);
    double dp = (fl + fr + ur - ul) / (dfl + dfr);
    double pn = ps - dp;
    if (pn < 1e-12) pn = 1e-12;
    double ch = 2.0 * fabs(pn - ps) / (pn + ps);
    ps = pn;
    if (ch < 1e-15) break;
  }
  double fl, dfl, fr, dfr;
  wave_curve(gamma, ps, rl, pl, cl, &fl, &dfl);
  wave_curve(gamma, ps, rr, pr, cr, &fr, &dfr);
  double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  if (pstar) *pstar = ps;
  if (ustar) *ustar = us;
  const double g1 = (gamma - 1.0) / (2.0 * gamma), g6 = (gamma - 1.0) / (gamma + 1.0);
  if (s <= us) {
    if (ps > pl) {
      double SL = ul - cl * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + g1);
      if (s <= SL) { *r = rl; *u = ul; *p = pl; }
      else { *r = rl * (ps / pl + g6) / (g6 * ps / pl + 1.0); *u = us; *p = ps; }
    } else {
      double SHL = ul - cl, cml = cl * pow(ps / pl, g1), STL = us - cml;
      if (s <= SHL) { *r = rl; *u = ul; *p = pl; }
      else if (s > STL) { *r = rl * pow(ps / pl, 1.0 / gamma); *u = us; *p = ps; }
      else {
        double uu = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * ul + s);
        double cc = 2.0 / (gamma + 1.0) * (cl + 0.5 * (gamma - 1.0) * (ul - s));
        *r = rl * pow(cc / cl, 2.0 / (gamma - 1.0));
        *u = uu;
        *p = pl * pow(cc / cl, 2.0 * gamma / (gamma - 1.0));
      }
    }
  } else {
    if (ps > pr) {
      double SR = ur + cr * sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + g1);
      if (s >= SR) { *r = rr; *u = ur; *p = pr; }
      else { *r = rr * (ps / pr + g6) / (g6 * ps / pr + 1.0); *u = us; *p = ps; }
    } else {
      double SHR = ur + cr, cmr = cr * pow(ps / pr, g1), STR = us + cmr;
      if (s >= SHR) { *r = rr; *u = ur; *p = pr; }
      else if (s < STR) { *r = rr * pow(ps / pr, 1.0 / gamma); *u = us; *p = ps; }
      else {
        double uu = 2.0 / (gamma + 1.0) * (-cr + 0.5 * (gamma - 1.0) * ur + s);
        double cc = 2.0 / (gamma + 1.0) * (cr - 0.5 * (gamma - 1.0) * (ur - s));
        *r = rr * pow(cc / cr, 2.0 / (gamma - 1.0));
        *u = uu;
        *p = pr * pow(cc / cr, 2.0 * gamma / (gamma - 1.0));
      }
    }
  }
  return 0;
}
