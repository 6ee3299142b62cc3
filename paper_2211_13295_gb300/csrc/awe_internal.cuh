// awe_internal.cuh -- device-side building blocks of the ADER-WENO zone update
// shared by the translation units of libawe.so.  Nothing here is part of the
// C ABI (include/awe.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/awe.h"
#include "fp_bits.cuh"

namespace awe {

constexpr int kMaxV = 5;

// ---------------------------------------------------------------------------
// Grid geometry passed by value to every kernel.
// Ghosted arrays: [var][z][y][x] with g = order ghost zones per side of every
// active dimension; "active-relative" coordinates run from -g to n+g-1.
// ---------------------------------------------------------------------------
struct Geo {
  int dim, N, g, nv;
  int n[3];        // active zones (n[2] = 1 in 2D)
  int G[3];        // ghosted extents (G[2] = 1 in 2D)
  long long ntot;  // ghosted zones per variable
  double dx[3], lo[3];
  double gamma, eps, cfl;
  double lin[4];
  int bc[6];
  double inflow[6][5];
  double pre[5];
  int fallback;  // positivity fallback of the face states
  int riemann;   // awe_riemann: Riemann solver of the corrector
  unsigned long long* fb_count;  // device counter of zones sent to the fallback (may be null)
  // the linear-weight reconstruction folded into one stencil per mode:
  // lst[a][j] = sum_k lin[k] c_k[a][j] on the differences d[j] (j = 0..2N)
  double lst[3][7];
  float lstf[3][7];
  float linf[4];   // lin in FP32 (the FP32 form's weights)
};

// index of an active-relative coordinate in a ghosted array
__host__ __device__ __forceinline__ long long gidx(const Geo& q, int i, int j, int k) {
  int gz = q.dim == 3 ? q.g : 0;
  return ((long long)(k + gz) * q.G[1] + (j + q.g)) * q.G[0] + (i + q.g);
}

// A rectangular region of zones in active-relative coordinates, [lo, lo+ext).
// r = (k e1 + j) e0 + i with 0 <= i < e0, 0 <= j < e1: unsigned 32-bit
// divisions while r fits in 32 bits (a 64-bit division is a long software
// sequence), 64-bit ones beyond
__host__ __device__ __forceinline__ void split3(long long r, int e0, int e1, int& i, int& j, int& k) {
  if (r >= 0 && r <= 0xffffffffLL) {
    const unsigned u = (unsigned)r, t = u / (unsigned)e0;
    i = (int)(u - t * (unsigned)e0);
    const unsigned kq = t / (unsigned)e1;
    j = (int)(t - kq * (unsigned)e1);
    k = (int)kq;
  } else {
    const long long t = r / e0;
    i = (int)(r - t * e0);
    const long long kq = t / e1;
    j = (int)(t - kq * e1);
    k = (int)kq;
  }
}

struct Region {
  int lo[3], ext[3];
  __host__ __device__ __forceinline__ long long size() const {
    return (long long)ext[0] * ext[1] * ext[2];
  }
  __host__ __device__ __forceinline__ long long index(int i, int j, int k) const {
    return ((long long)(k - lo[2]) * ext[1] + (j - lo[1])) * ext[0] + (i - lo[0]);
  }
  __host__ __device__ __forceinline__ void coords(long long r, int& i, int& j, int& k) const {
    split3(r, ext[0], ext[1], i, j, k);
    i += lo[0];
    j += lo[1];
    k += lo[2];
  }
};

// ---------------------------------------------------------------------------
// mode counts
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int binom_c(int n, int k) {
  return k == 0 ? 1 : binom_c(n - 1, k - 1) * n / k;
}
template <int D, int N> struct Modes {
  static constexpr int NS = binom_c(N + D, D);          // spatial modes, degree <= N
  static constexpr int NG = binom_c(N - 1 + D + 1, D + 1);  // space-time, degree <= N-1
  static constexpr int NV = D + 2;
  static constexpr int NN = N + 1;                       // predictor nodes per dimension
  static constexpr int NSN = D == 2 ? NN * NN : NN * NN * NN;  // spatial nodes
  static constexpr int NQ = (N + 2) / 2;                 // face Gauss points per dimension
  static constexpr int NFQ = D == 2 ? NQ * NQ : NQ * NQ * NQ;  // face quadrature points
};

// ---------------------------------------------------------------------------
// Euler equations, ideal gas
// ---------------------------------------------------------------------------
// Division and square root of the FP32 form's predictor and Riemann fluxes:
// the fast forms (__fdividef: within 2 ulp for a divisor of magnitude in
// [2^-126, 2^126]; x rsqrtf(x): within 3 ulp for x > 0, 0 at 0, NaN below)
// instead of the IEEE refinement sequences.  FP64 keeps the IEEE operations.
template <typename T> __device__ __forceinline__ T fdiv(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fdividef(a, b);
  else return a / b;
}
template <typename T> __device__ __forceinline__ T fsqrt(T x) {
  if constexpr (sizeof(T) == 4) {
    const float inf = __int_as_float(0x7f800000);
    return x > 0.f ? (x < inf ? x * rsqrtf(x) : x) : x == 0.f ? 0.f : __int_as_float(0x7fffffff);
  } else {
    return sqrt(x);
  }
}

template <int D, typename T>
__device__ __forceinline__ T pressure_of(const T* U, T gm1) {
  T irho = T(1) / U[0];
  T m2 = U[1] * U[1];
#pragma unroll
  for (int d = 1; d < D; ++d) m2 = fma(U[1 + d], U[1 + d], m2);
  return gm1 * (U[D + 1] - T(0.5) * m2 * irho);
}

// Physical fluxes of all D directions at one state (shared 1/rho and p).
template <int D, typename T>
__device__ __forceinline__ void phys_fluxes_irho(const T* U, T irho, T gm1, T F[D][D + 2]) {
  T v[D];
#pragma unroll
  for (int d = 0; d < D; ++d) v[d] = U[1 + d] * irho;
  T m2 = U[1] * v[0];
#pragma unroll
  for (int d = 1; d < D; ++d) m2 = fma(U[1 + d], v[d], m2);
  T p = gm1 * (U[D + 1] - T(0.5) * m2);
  T Ep = U[D + 1] + p;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    F[d][0] = U[1 + d];
#pragma unroll
    for (int e = 0; e < D; ++e) F[d][1 + e] = U[1 + e] * v[d];
    F[d][1 + d] += p;
    F[d][D + 1] = Ep * v[d];
  }
}
template <int D, typename T>
__device__ __forceinline__ void phys_fluxes(const T* U, T gm1, T F[D][D + 2]) {
  phys_fluxes_irho<D, T>(U, fdiv(T(1), U[0]), gm1, F);
}
// 1/a and 1/b from one division: 1/a = b / (ab), 1/b = a / (ab) (densities of
// a pair of nodes; ab stays far inside the range for physical densities)
template <typename T>
__device__ __forceinline__ void recip_pair(T a, T b, T& ia, T& ib) {
  const T r = fdiv(T(1), a * b);
  ia = b * r;
  ib = a * r;
}

// HLLC flux across a face normal to direction dir (Toro, Spruce & Speares):
// Davis-Einfeldt wave speeds with Roe averages, S* from the pressure
// balance, left star state when S* = 0.
template <int D, typename T>
__device__ __forceinline__ void hllc(const T* UL, const T* UR, int dir, T gamma, T* F) {
  const T gm1 = gamma - T(1);
  T rl = UL[0], rr = UR[0];
  T irl, irr;
  recip_pair<T>(rl, rr, irl, irr);
  T vl[D], vr[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vl[d] = UL[1 + d] * irl;
    vr[d] = UR[1 + d] * irr;
  }
  T kl = UL[1] * vl[0], kr = UR[1] * vr[0];
#pragma unroll
  for (int d = 1; d < D; ++d) {
    kl = fma(UL[1 + d], vl[d], kl);
    kr = fma(UR[1 + d], vr[d], kr);
  }
  T El = UL[D + 1], Er = UR[D + 1];
  T pl = gm1 * (El - T(0.5) * kl), pr = gm1 * (Er - T(0.5) * kr);
  T cl = fsqrt(gamma * pl * irl), cr = fsqrt(gamma * pr * irr);
  T ul = vl[dir], ur = vr[dir];
  T sl = fsqrt(rl), sr = fsqrt(rr);
  T iden = fdiv(T(1), sl + sr);
  T vt2 = T(0), vtn = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    T vt = (sl * vl[d] + sr * vr[d]) * iden;
    vt2 = fma(vt, vt, vt2);
    if (d == dir) vtn = vt;
  }
  T Ht = (sl * (El + pl) * irl + sr * (Er + pr) * irr) * iden;
  T ct = fsqrt(gm1 * (Ht - T(0.5) * vt2));
  T SL = fmin(ul - cl, vtn - ct);
  T SR = fmax(ur + cr, vtn + ct);
  T ml = rl * (SL - ul), mr = rr * (SR - ur);
  T Ss = fdiv(pr - pl + ul * ml - ur * mr, ml - mr);
  // branches in the order F_L (0 <= S_L), F*_L (0 <= S*), F*_R (0 < S_R), F_R
  if (T(0) <= SL) {
    F[0] = UL[1 + dir];
#pragma unroll
    for (int e = 0; e < D; ++e) F[1 + e] = UL[1 + e] * ul;
    F[1 + dir] += pl;
    F[D + 1] = (El + pl) * ul;
  } else if (!(T(0) <= Ss) && !(T(0) < SR)) {
    F[0] = UR[1 + dir];
#pragma unroll
    for (int e = 0; e < D; ++e) F[1 + e] = UR[1 + e] * ur;
    F[1 + dir] += pr;
    F[D + 1] = (Er + pr) * ur;
  } else {
    const bool left = T(0) <= Ss;
    const T* U = left ? UL : UR;
    T S = left ? SL : SR, u = left ? ul : ur, m = left ? ml : mr, p = left ? pl : pr;
    T rho = left ? rl : rr, E = left ? El : Er, ir = left ? irl : irr;
    T f = fdiv(m, S - Ss);
    // F* = F(U) + S (U* - U)
    F[0] = U[1 + dir] + S * (f - rho);
#pragma unroll
    for (int e = 0; e < D; ++e) {
      T us = (e == dir) ? f * Ss : f * (U[1 + e] * ir);
      F[1 + e] = U[1 + e] * u + S * (us - U[1 + e]);
    }
    F[1 + dir] += p;
    T Es = f * (E * ir + (Ss - u) * (Ss + fdiv(p, m)));
    F[D + 1] = (E + p) * u + S * (Es - E);
  }
}

// Physical flux along dir of a conserved state whose velocities, pressure
// and energy are already known.
template <int D, typename T>
__device__ __forceinline__ void dir_flux(const T* U, const T* v, T p, int dir, T* F) {
  const T un = v[dir];
  F[0] = U[1 + dir];
#pragma unroll
  for (int e = 0; e < D; ++e) F[1 + e] = U[1 + e] * un;
  F[1 + dir] += p;
  F[D + 1] = (U[D + 1] + p) * un;
}

// HLL and HLLEM (the other solvers of Sec. I.1 besides HLLC and Rusanov).
// HLL: the single state between the Davis-Einfeldt speeds of hllc();
// F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) inside the fan.
// HLLEM (EM = true): the jump term loses delta * sum_k a_k r_k over the
// linearly degenerate Roe waves (the contact, a_c = drho - dp/c~^2,
// r_c = (1, v~, |v~|^2/2); each shear wave t, a_t = rho~ dv_t,
// r_t = (0, e_t, v~_t)), delta = 1 - min(u~,0)/S_L - max(u~,0)/S_R, which
// resolves isolated contacts and shear waves exactly.
template <int D, typename T, bool EM>
__device__ __forceinline__ void hll_family(const T* UL, const T* UR, int dir, T gamma, T* F) {
  constexpr int NV = D + 2;
  const T gm1 = gamma - T(1);
  T rl = UL[0], rr = UR[0];
  T irl, irr;
  recip_pair<T>(rl, rr, irl, irr);
  T vl[D], vr[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vl[d] = UL[1 + d] * irl;
    vr[d] = UR[1 + d] * irr;
  }
  T kl = UL[1] * vl[0], kr = UR[1] * vr[0];
#pragma unroll
  for (int d = 1; d < D; ++d) {
    kl = fma(UL[1 + d], vl[d], kl);
    kr = fma(UR[1 + d], vr[d], kr);
  }
  T El = UL[D + 1], Er = UR[D + 1];
  T pl = gm1 * (El - T(0.5) * kl), pr = gm1 * (Er - T(0.5) * kr);
  T cl = fsqrt(gamma * pl * irl), cr = fsqrt(gamma * pr * irr);
  T ul = vl[dir], ur = vr[dir];
  T sl = fsqrt(rl), sr = fsqrt(rr);
  T iden = fdiv(T(1), sl + sr);
  T vt[D], vt2 = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vt[d] = (sl * vl[d] + sr * vr[d]) * iden;
    vt2 = fma(vt[d], vt[d], vt2);
  }
  T Ht = (sl * (El + pl) * irl + sr * (Er + pr) * irr) * iden;
  T ct = fsqrt(gm1 * (Ht - T(0.5) * vt2));
  T SL = fmin(ul - cl, vt[dir] - ct);
  T SR = fmax(ur + cr, vt[dir] + ct);
  if (T(0) <= SL) {
    dir_flux<D, T>(UL, vl, pl, dir, F);
    return;
  }
  if (SR <= T(0)) {
    dir_flux<D, T>(UR, vr, pr, dir, F);
    return;
  }
  T FL[NV], FR[NV], jump[NV];
  dir_flux<D, T>(UL, vl, pl, dir, FL);
  dir_flux<D, T>(UR, vr, pr, dir, FR);
#pragma unroll
  for (int s = 0; s < NV; ++s) jump[s] = UR[s] - UL[s];
  if (EM) {
    const T ut = vt[dir];
    const T delta = T(1) - fdiv(fmin(ut, T(0)), SL) - fdiv(fmax(ut, T(0)), SR);
    const T ac = delta * ((rr - rl) - fdiv(pr - pl, ct * ct));
    jump[0] -= ac;
#pragma unroll
    for (int e = 0; e < D; ++e) jump[1 + e] -= ac * vt[e];
    jump[D + 1] -= ac * (T(0.5) * vt2);
    const T rt = sl * sr;
#pragma unroll
    for (int t = 0; t < D; ++t) {
      if (t == dir) continue;
      const T at = delta * (rt * (vr[t] - vl[t]));
      jump[1 + t] -= at;
      jump[D + 1] -= at * vt[t];
    }
  }
  const T inv = fdiv(T(1), SR - SL), slsr = SL * SR;
#pragma unroll
  for (int s = 0; s < NV; ++s) F[s] = (SR * FL[s] - SL * FR[s] + slsr * jump[s]) * inv;
}

// Rusanov (local Lax-Friedrichs): (F_L + F_R)/2 - S (U_R - U_L)/2 with
// S = max(|u_L| + c_L, |u_R| + c_R), u the velocity normal to the face.
template <int D, typename T>
__device__ __forceinline__ void rusanov(const T* UL, const T* UR, int dir, T gamma, T* F) {
  constexpr int NV = D + 2;
  const T gm1 = gamma - T(1);
  T irl, irr;
  recip_pair<T>(UL[0], UR[0], irl, irr);
  T vl[D], vr[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    vl[d] = UL[1 + d] * irl;
    vr[d] = UR[1 + d] * irr;
  }
  T kl = UL[1] * vl[0], kr = UR[1] * vr[0];
#pragma unroll
  for (int d = 1; d < D; ++d) {
    kl = fma(UL[1 + d], vl[d], kl);
    kr = fma(UR[1 + d], vr[d], kr);
  }
  T pl = gm1 * (UL[D + 1] - T(0.5) * kl), pr = gm1 * (UR[D + 1] - T(0.5) * kr);
  T S = fmax(fabs(vl[dir]) + fsqrt(gamma * pl * irl), fabs(vr[dir]) + fsqrt(gamma * pr * irr));
  T FL[NV], FR[NV];
  dir_flux<D, T>(UL, vl, pl, dir, FL);
  dir_flux<D, T>(UR, vr, pr, dir, FR);
#pragma unroll
  for (int s = 0; s < NV; ++s) F[s] = T(0.5) * (FL[s] + FR[s]) - T(0.5) * S * (UR[s] - UL[s]);
}

// The corrector's Riemann solver, chosen at compile time (K = awe_riemann).
template <int K, int D, typename T>
__device__ __forceinline__ void riemann(const T* UL, const T* UR, int dir, T gamma, T* F) {
  if constexpr (K == 1) hll_family<D, T, false>(UL, UR, dir, gamma, F);
  else if constexpr (K == 2) hll_family<D, T, true>(UL, UR, dir, gamma, F);
  else if constexpr (K == 3) rusanov<D, T>(UL, UR, dir, gamma, F);
  else hllc<D, T>(UL, UR, dir, gamma, F);
}

// rho > 0, p > 0 and every component finite (positivity fallback test)
template <int D, typename T>
__device__ __forceinline__ bool state_physical(const T* U, T gm1) {
  bool ok = U[0] > T(0);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) ok = ok && isfinite(U[v]);
  T m2 = U[1] * U[1];
#pragma unroll
  for (int d = 1; d < D; ++d) m2 = fma(U[1 + d], U[1 + d], m2);
  T p = gm1 * (U[D + 1] - T(0.5) * m2 / U[0]);
  return ok && p > T(0);
}

// Signal speed max_d (|v_d| + c)/dx_d of one zone (FP64), and physicality.
template <int D>
__device__ __forceinline__ double zone_signal(const double* U, double gamma, const double* idx_,
                                              bool& ok) {
  double rho = U[0];
  double irho = 1.0 / rho;
  double m2 = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) m2 = fma(U[1 + d], U[1 + d], m2);
  double p = (gamma - 1.0) * (U[D + 1] - 0.5 * m2 * irho);
  ok = (rho > 0.0) && (p > 0.0);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) ok = ok && isfinite(U[v]);
  double c = sqrt(gamma * p * irho);
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) s = fmax(s, (fabs(U[1 + d] * irho) + c) * idx_[d]);
  return s;
}

// ---------------------------------------------------------------------------
// WENO 1D in the "difference" form: d[j] = u(j-N) - u(0), j = 0..2N.
// Candidates, smoothness and the final combination in T; the epsilon and
// weight path in FP64 (product form: omega_k ~ lin_k prod_{j!=k} (eps+beta_j)^2,
// which equals lin_k/(eps+beta_k)^2 normalised).
// ---------------------------------------------------------------------------
#include "stencils.inc"

// Order 2: the paper's MC limiter (Fig. 3), slope from the one-sided
// differences a = u(i+1)-u(i), b = u(i)-u(i-1):
// min(|a+b|/2, cfac|a|, cfac|b|) * (sgn(a)/2 + sgn(b)/2), sgn(0) = +1;
// compression factor 2.0 for the density, 1.5 for the other variables.
template <typename T>
__device__ __forceinline__ T mc_slope(T a, T b, T cfac) {
  T m = fmin(T(0.5) * fabs(a + b), fmin(cfac * fabs(a), cfac * fabs(b)));
  T sa = a >= T(0) ? T(0.5) : T(-0.5), sb = b >= T(0) ? T(0.5) : T(-0.5);
  return m * (sa + sb);
}

template <int N, typename T>
__device__ __forceinline__ void weno_candidates(const T* d, T c[N + 1][N]) {
  if constexpr (N == 2) weno_candidates_n2<T>(d, c);
  else weno_candidates_n3<T>(d, c);
}

template <int N, typename T>
__device__ __forceinline__ T weno_beta(const T* c) {
  if constexpr (N == 2) {
    return c[0] * c[0] + T(13.0 / 3.0) * (c[1] * c[1]);
  } else {
    T a = fma(T(0.1), c[2], c[0]);
    return a * a + T(13.0 / 3.0) * (c[1] * c[1]) + T(781.0 / 20.0) * (c[2] * c[2]);
  }
}

// Nonlinear weights (FP64) from the smoothness indicators.
template <int N>
__device__ __forceinline__ void weno_weights(const double* beta, const double* lin, double eps,
                                             double* om) {
  double s[N + 1];
#pragma unroll
  for (int k = 0; k <= N; ++k) {
    double t = eps + beta[k];
    s[k] = t * t;
  }
  double P[N + 1];
  if constexpr (N == 2) {
    P[0] = lin[0] * (s[1] * s[2]);
    P[1] = lin[1] * (s[0] * s[2]);
    P[2] = lin[2] * (s[0] * s[1]);
  } else {
    double s01 = s[0] * s[1], s23 = s[2] * s[3];
    P[0] = lin[0] * (s[1] * s23);
    P[1] = lin[1] * (s[0] * s23);
    P[2] = lin[2] * (s[3] * s01);
    P[3] = lin[3] * (s[2] * s01);
  }
  double sum = P[0];
#pragma unroll
  for (int k = 1; k <= N; ++k) sum += P[k];
  double inv = 1.0 / sum;
#pragma unroll
  for (int k = 0; k <= N; ++k) om[k] = P[k] * inv;
}

// Full 1D WENO: modal coefficients out[0..N-1] of modes 1..N.
// The linear-weight reconstruction as one folded stencil per mode (2N terms):
// the same linear combination of the candidates, in a single pass.
template <int N, typename T>
__device__ __forceinline__ void linear1d(const T* d, const T (*lst)[7], T* out) {
#pragma unroll
  for (int a = 0; a < N; ++a) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j <= 2 * N; ++j)
      if (j != N) acc = fma(lst[a][j], d[j], acc);
    out[a] = acc;
  }
}

template <int N, typename T>
__device__ __forceinline__ void weno1d(const T* d, const double* lin, const float* linf, double eps,
                                       bool linear, T* out) {
  T c[N + 1][N];
  weno_candidates<N, T>(d, c);
  if constexpr (sizeof(T) == 4) {
    if (!linear) {
      // FP32 form: the epsilon path, t_k = eps + beta_k, in FP64 (beta_k
      // widened exactly, t_k narrowed toward zero, both by bit operations:
      // fp_bits.cuh); the weights lin_k / t_k^2, normalised, in FP32 with
      // the fast reciprocal (t_k >= eps = 1e-12, so lin_k / t_k^2 <= 1e24;
      // for t_k above ~1e19 the term underflows, as the IEEE form's t_k^2
      // overflows)
      float q[N + 1], sum = 0.f;
#pragma unroll
      for (int k = 0; k <= N; ++k) {
        const float t = f64_to_f32_rz(eps + nonneg_f32_to_f64(weno_beta<N, T>(c[k])));
        const float u = __fdividef(1.f, t);
        q[k] = linf[k] * (u * u);
        sum += q[k];
      }
      const float inv = __fdividef(1.f, sum);
#pragma unroll
      for (int a = 0; a < N; ++a) {
        float acc = (q[0] * inv) * c[0][a];
#pragma unroll
        for (int k = 1; k <= N; ++k) acc = fmaf(q[k] * inv, c[k][a], acc);
        out[a] = acc;
      }
      return;
    }
  }
  double om[N + 1];
  if (linear) {
#pragma unroll
    for (int k = 0; k <= N; ++k) om[k] = lin[k];
  } else {
    double beta[N + 1];
#pragma unroll
    for (int k = 0; k <= N; ++k) beta[k] = (double)weno_beta<N, T>(c[k]);
    weno_weights<N>(beta, lin, eps, om);
  }
#pragma unroll
  for (int a = 0; a < N; ++a) {
    T acc = T(om[0]) * c[0][a];
#pragma unroll
    for (int k = 1; k <= N; ++k) acc = fma(T(om[k]), c[k][a], acc);
    out[a] = acc;
  }
}

// ---------------------------------------------------------------------------
// Predictor tables (host-computed from closed forms, uploaded at create).
// Nodes: Gauss-Legendre with NN = N+1 points on [-1/2,1/2] (space) and
// [0,1] (time); face points: 2-point Gauss-Legendre.
// ---------------------------------------------------------------------------
template <typename T> struct Tabs {
  T PN[4][4];        // P_a(x_i)
  T WPN[4][4];       // w_i P_a(x_i) / |P_a|^2
  T QN[4][4][4];     // w_i sum_{a'=a+1}^{a+s} D[a'][a] P_a'(x_i) / |P_a'|^2  [a][s][i]
  T IT[4][4];        // I_e(tau_t) = int_0^tau_t L_e
  T WLT[4][4];       // w_t L_e(tau_t) / |L_e|^2
  T PF[4][2];        // P_a at the two face points
  T PE[4][2];        // P_a(-1/2), P_a(+1/2)
  T ITF[4][2];       // I_e at the two face time points
  T WF[2];           // face weights
};

// Each translation unit that reads the tables holds its own constant copy
// (no relocatable device code); build_tabs (awe_tables.cu) fills host copies
// and UPLOAD_LOCAL_TABLES() copies them into the calling unit's symbols.
void build_tabs(Tabs<double>* td, Tabs<float>* tf);  // [3] each, N = 1, 2, 3
static __constant__ Tabs<double> c_tab_d[3];
static __constant__ Tabs<float> c_tab_f[3];
template <typename T> __device__ __forceinline__ const Tabs<T>& tabs(int N);
template <> __device__ __forceinline__ const Tabs<double>& tabs<double>(int N) { return c_tab_d[N - 1]; }
template <> __device__ __forceinline__ const Tabs<float>& tabs<float>(int N) { return c_tab_f[N - 1]; }
static inline cudaError_t upload_local_tables(cudaStream_t s) {
  Tabs<double> td[3];
  Tabs<float> tf[3];
  build_tabs(td, tf);
  cudaError_t e = cudaMemcpyToSymbolAsync(c_tab_d, td, sizeof(td), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_tab_f, tf, sizeof(tf), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// ---------------------------------------------------------------------------
// Host-side launchers (one per stage), defined in the stage files.
// ---------------------------------------------------------------------------
struct Bufs;  // defined in awe_api.cu


// ghost zones of U at time *d_t + c * *d_dt (c = 0: *d_t; d_dt may then be null)
void launch_fill_ghosts(const Geo& q, double* U, const double* d_t, const double* d_dt, double c,
                        cudaStream_t s);
void launch_set_scalar(double* p, double v, cudaStream_t s);
long long halo_count(const Geo& q);
// a posteriori fallback (awe_flux.cu)
void launch_store_fluxes(const Geo& q, int prec, const void* F, int z0, int z1, double* Ffull, cudaStream_t s);
void launch_fb_passes(const Geo& q, const double* Uold, double* Unew, const double* Ffull, unsigned char* flags,
                      const double* d_dt, int passes, cudaStream_t s);
constexpr int kFallbackPasses = 4;
void launch_halo(const Geo& q, double* U, int side, double* buf, bool pack, cudaStream_t s);
void launch_signal_max(const Geo& q, const double* U, unsigned long long* smax, int* err,
                       cudaStream_t s);
void launch_finalize(const Geo& q, double* d_t, double* d_dt, unsigned long long* smax,
                     int advance, cudaStream_t s);

// reconstruction passes; fields in T (double or float)
void launch_recon(const Geo& q, int prec, const double* U, const unsigned char* flags, int z0,
                  int z1, void* X, void* Y, void* XY, void* W, cudaStream_t s,
                  cudaEvent_t* ev /* 3 events or nullptr */);
void launch_predict(const Geo& q, int prec, int picard, const void* W, const double* d_dt,
                    int z0, int z1, void* FS, cudaStream_t s);
void launch_flux(const Geo& q, int prec, const void* FS, int z0, int z1, void* F, cudaStream_t s);
void launch_update(const Geo& q, int prec, const double* Uold, const void* F, const double* d_dt,
                   int z0, int z1, double* Unew, unsigned long long* smax, int* err,
                   cudaStream_t s);

// regions of the reconstruction passes for the slab [z0, z1)
Region region_x(const Geo& q, int z0, int z1);
Region region_y(const Geo& q, int z0, int z1);
Region region_box(const Geo& q, int z0, int z1);

}  // namespace awe
