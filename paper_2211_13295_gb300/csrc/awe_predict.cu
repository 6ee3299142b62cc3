// awe_predict.cu -- ADER predictor (the paper's Predictor / Predictor_Ptwise,
// Fig. 4) and the evaluation of each zone's space-time polynomial at its face
// quadrature points (the face values of Make_Flux_X/Y/Z, Fig. 5).
//
// Predictor (local space-time Picard iteration):
//   q^0 = w(xi),  q^{k+1} = w - int_0^tau G^k,  G^k = sum_d (dt/dx_d) d/dxi_d Pi_N F_d(q^k),
// with Pi_N the L2 projection onto space-time polynomials of total degree <= N
// taken with tensor Gauss-Legendre quadrature of N+1 nodes per dimension.  G^k
// has total degree <= N-1, so each sweep only needs its NG coefficients g:
//   g_beta = sum_d lam_d sum_nodes F_d(node) K^d_beta(node),
// K^d_beta = weights * [sum_{a'>beta_d} D[a'][beta_d] P_a'/|P_a'|^2](xi_d)
//            * prod_{o != d} P_{beta_o}/|P_{beta_o}|^2 * L_{beta_t}/|L_{beta_t}|^2,
// where the a' range is limited by the total degree N.  Sweep 0 sees a
// time-independent flux, so only beta_t = 0 coefficients are non-zero and the
// flux is evaluated at the spatial nodes only.
//
// Two implementations with the same arithmetic content:
//  * direct: one thread per zone, node tables in memory (orders 3 in 2D/3D,
//    order 4 in 2D);
//  * factorised: one warp per zone, shared memory, tensor contractions one
//    dimension at a time (order 4 in 3D, ~2.5x fewer FP64 operations).
#include "awe_internal.cuh"
#include "awe_tables.h"
#include "predict_index.cuh"

namespace awe {

// ---------------------------------------------------------------------------
// direct predictor
// ---------------------------------------------------------------------------
// whether space-time mode b (degree <= N-1, time exponent outermost) has an
// odd time exponent
template <int D, int N> __host__ __device__ constexpr bool st_time_odd(int b) {
  int idx = 0;
  for (int e = 0; e <= N - 1; ++e) {
    const int K = N - 1 - e;
    const int cnt = D == 3 ? (K + 1) * (K + 2) * (K + 3) / 6 : (K + 1) * (K + 2) / 2;
    if (b < idx + cnt) return (e & 1) != 0;
    idx += cnt;
  }
  return false;
}

// compile-time positions in the mode enumerations of the tables: spatial
// modes (a, b, c) of total degree <= N with c outermost, then b, then a;
// space-time modes (a, b, c, e) of total degree <= M with e outermost
template <int D, int N> __host__ __device__ constexpr int sp_index(int a, int b, int c) {
  int idx = 0;
  for (int cc = 0; cc <= (D == 3 ? N : 0); ++cc)
    for (int bb = 0; bb <= N - cc; ++bb)
      for (int aa = 0; aa <= N - bb - cc; ++aa) {
        if (aa == a && bb == b && cc == c) return idx;
        ++idx;
      }
  return -1;
}
template <int D, int M> __host__ __device__ constexpr int st_index(int a, int b, int c, int e) {
  int idx = 0;
  for (int ee = 0; ee <= M; ++ee)
    for (int cc = 0; cc <= (D == 3 ? M - ee : 0); ++cc)
      for (int bb = 0; bb <= M - ee - cc; ++bb)
        for (int aa = 0; aa <= M - ee - bb - cc; ++aa) {
          if (aa == a && bb == b && cc == c && ee == e) return idx;
          ++idx;
        }
  return -1;
}
// exponent k (0 = a, 1 = b, 2 = c, 3 = e) of space-time mode i
template <int D, int M> __host__ __device__ constexpr int st_exp(int i, int k) {
  int idx = 0;
  for (int ee = 0; ee <= M; ++ee)
    for (int cc = 0; cc <= (D == 3 ? M - ee : 0); ++cc)
      for (int bb = 0; bb <= M - ee - cc; ++bb)
        for (int aa = 0; aa <= M - ee - bb - cc; ++aa) {
          if (idx == i) return k == 0 ? aa : k == 1 ? bb : k == 2 ? cc : ee;
          ++idx;
        }
  return -1;
}

// Mass row of the new G (thread-per-zone form).  The mass flux of direction d
// is the momentum q_{1+d} = w_{1+d} - sum_g g_{1+d} P P (P) I_e(tau), of total
// degree <= N: the N+1-point Gauss rules integrate its products with the test
// functions exactly, so its projection is itself and the G coefficient is its
// exact derivative, from I_0 = (L_0 + L_1)/2, I_e = (L_{e+1} - L_{e-1}) /
// (2(2e+1)) and dP1 = P0, dP2 = 2 P1, dP3 = 3 P2 + P0/10.  Same value as
// projecting the node fluxes, up to rounding, without the node work.
template <int D, int N, typename T>
__device__ __forceinline__ T mass_gmode_direct(const T (*w)[Modes<D, N>::NS], const T (*g)[Modes<D, N>::NG],
                                               const T* lam, int b) {
  const int e = st_exp<D, N - 1>(b, 3);
  T acc = T(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      int ix[3] = {st_exp<D, N - 1>(b, 0), st_exp<D, N - 1>(b, 1), D == 3 ? st_exp<D, N - 1>(b, 2) : 0};
      const int ad = ix[d];
      if (k == 1 && ad != 0) break;
      ix[d] = k == 0 ? ad + 1 : 3;
      const int deg = ix[0] + ix[1] + ix[2];
      if (deg + e > N) continue;
      const T f = k == 0 ? T(ad + 1) : T(0.1);   // coefficient of P_ad in dP_{a'}
      // coefficient of L_e of the momentum's mode ix
      T gg[3];
#pragma unroll
      for (int ee = 0; ee < 3; ++ee)
        gg[ee] = deg + ee <= N - 1 ? g[1 + d][st_index<D, N - 1>(ix[0], ix[1], ix[2], ee)] : T(0);
      T m;
      if (e == 0) m = fma(T(1.0 / 6.0), gg[1], fma(T(-0.5), gg[0], w[1 + d][sp_index<D, N>(ix[0], ix[1], ix[2])]));
      else if (e == 1) m = fma(T(0.1), gg[2], T(-0.5) * gg[0]);
      else m = T(-1.0 / 6.0) * gg[1];
      s = fma(f, m, s);
    }
    acc = fma(lam[d], s, acc);
  }
  return acc;
}

template <int D, int N, typename T>
__global__ void __launch_bounds__(128) k_predict_direct(Geo q, Region box, const T* __restrict__ W,
                                                        const double* __restrict__ d_dt, int picard,
                                                        const T* __restrict__ tab, PTabLayout L,
                                                        T* __restrict__ FS) {
  using M = Modes<D, N>;
  constexpr int NV = M::NV, NS = M::NS, NG = M::NG, NN = M::NN, NSN = M::NSN, NFQ = M::NFQ;
  constexpr int NG0 = Modes<D, N - 1>::NS;  // G-modes with beta_t = 0 come first
  const long long nb = box.size();
  const double dt = *d_dt;
  T lam[D];
#pragma unroll
  for (int d = 0; d < D; ++d) lam[d] = (T)(dt / q.dx[d]);
  const T gm1 = (T)(q.gamma - 1.0);
  const T* EV = tab + L.ev;
  const T* KP = tab + L.kp;
  const T* KS = tab + L.ks;
  const T* WS = tab + L.ws;
  const T* FW = tab + L.fw;
  const T* FG = tab + L.fg;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nb;
       r += (long long)gridDim.x * blockDim.x) {
    T w[NV][NS];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int m = 0; m < NS; ++m) w[v][m] = W[((long long)v * NS + m) * nb + r];
    T g[NV][NG];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int b = 0; b < NG; ++b) g[v][b] = T(0);
    if (picard >= 1) {
      // sweep 0: time-independent flux at the spatial nodes (momentum and
      // energy rows; the mass row from the momentum's coefficients, g = 0)
#pragma unroll
      for (int b = 0; b < NG0; ++b) g[0][b] = mass_gmode_direct<D, N, T>(w, g, lam, b);
      for (int s = 0; s < NSN; ++s) {
        T qn[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T acc = T(0);
#pragma unroll
          for (int m = 0; m < NS; ++m) acc = fma(w[v][m], WS[s * NS + m], acc);
          qn[v] = acc;
        }
        T F[D][D + 2];
        phys_fluxes<D, T>(qn, gm1, F);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const T* ks = KS + ((long long)d * NSN + s) * NG;
#pragma unroll
          for (int v = 1; v < NV; ++v) {
            T f = lam[d] * F[d][v];
#pragma unroll
            for (int b = 0; b < NG0; ++b) g[v][b] = fma(f, ks[b], g[v][b]);
          }
        }
      }
      for (int sweep = 1; sweep < picard; ++sweep) {
        T gn[NV][NG];
#pragma unroll
        for (int b = 0; b < NG; ++b) gn[0][b] = mass_gmode_direct<D, N, T>(w, g, lam, b);
#pragma unroll
        for (int v = 1; v < NV; ++v)
#pragma unroll
          for (int b = 0; b < NG; ++b) gn[v][b] = T(0);
        for (int s = 0; s < NSN; ++s) {
          T wn[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < NS; ++m) acc = fma(w[v][m], WS[s * NS + m], acc);
            wn[v] = acc;
          }
          // time nodes in symmetric pairs (t, NN-1-t): the projection kernel of
          // the second is (-1)^e times that of the first (symmetric weights,
          // L_e(1 - tau) = (-1)^e L_e(tau)), so a pair enters through the sum
          // of its fluxes (even e) or their difference (odd e); with NN odd
          // the middle node enters alone
#pragma unroll
          for (int t = 0; t < (NN + 1) / 2; ++t) {
            const int t2 = NN - 1 - t;
            T Fa[D][D + 2], Fb[D][D + 2];
            T qn[2][NV];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (h == 1 && t2 == t) break;
              const int node = s * NN + (h ? t2 : t);
              const T* ev = EV + (long long)node * NG;
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                T acc = wn[v];
#pragma unroll
                for (int b = 0; b < NG; ++b) acc = fma(-g[v][b], ev[b], acc);
                qn[h][v] = acc;
              }
            }
            if (t2 != t) {
              T ia, ib;
              recip_pair<T>(qn[0][0], qn[1][0], ia, ib);
              phys_fluxes_irho<D, T>(qn[0], ia, gm1, Fa);
              phys_fluxes_irho<D, T>(qn[1], ib, gm1, Fb);
            } else {
              phys_fluxes<D, T>(qn[0], gm1, Fa);
            }
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const T* kp = KP + ((long long)d * (NSN * NN) + s * NN + t) * NG;
#pragma unroll
              for (int v = 1; v < NV; ++v) {
                const T fs = t2 != t ? lam[d] * (Fa[d][v] + Fb[d][v]) : lam[d] * Fa[d][v];
                const T fd = t2 != t ? lam[d] * (Fa[d][v] - Fb[d][v]) : fs;
#pragma unroll
                for (int b = 0; b < NG; ++b) gn[v][b] = fma(st_time_odd<D, N>(b) ? fd : fs, kp[b], gn[v][b]);
              }
            }
          }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
          for (int b = 0; b < NG; ++b) g[v][b] = gn[v][b];
      }
    }
    // face quadrature states: q = w(face point) - int_0^tau G; with the
    // positivity fallback, a first pass checks every face point and a zone
    // with a non-physical one writes its mean instead
    // Rows (d, side, point) with point = sp + NSP * it: the w part depends on
    // the spatial point sp only, so it is formed once for the NQ time points.
    constexpr int NSP = NFQ / M::NQ;   // spatial points per face
    bool bad = false;
    if (q.fallback) {
      for (int ds = 0; ds < D * 2; ++ds)
        for (int sp = 0; sp < NSP; ++sp) {
          const T* fw = FW + (long long)(ds * NFQ + sp) * NS;
          T wv[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T acc = T(0);
#pragma unroll
            for (int m = 0; m < NS; ++m) acc = fma(w[v][m], fw[m], acc);
            wv[v] = acc;
          }
#pragma unroll
          for (int it = 0; it < M::NQ; ++it) {
            const T* fg = FG + (long long)(ds * NFQ + sp + NSP * it) * NG;
            T u[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              T acc = wv[v];
#pragma unroll
              for (int b = 0; b < NG; ++b) acc = fma(-g[v][b], fg[b], acc);
              u[v] = acc;
            }
            bad = bad || !state_physical<D, T>(u, gm1);
          }
        }
      if (bad && q.fb_count) atomicAdd(q.fb_count, 1ULL);
    }
    for (int ds = 0; ds < D * 2; ++ds)
      for (int sp = 0; sp < NSP; ++sp) {
        const T* fw = FW + (long long)(ds * NFQ + sp) * NS;
        T wv[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T acc = T(0);
#pragma unroll
          for (int m = 0; m < NS; ++m) acc = fma(w[v][m], fw[m], acc);
          wv[v] = acc;
        }
#pragma unroll
        for (int it = 0; it < M::NQ; ++it) {
          const int row = ds * NFQ + sp + NSP * it;
          const T* fg = FG + (long long)row * NG;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T acc = wv[v];
#pragma unroll
            for (int b = 0; b < NG; ++b) acc = fma(-g[v][b], fg[b], acc);
            FS[((long long)row * NV + v) * nb + r] = bad ? w[v][0] : acc;
          }
        }
      }
  }
}

// ---------------------------------------------------------------------------
// factorised predictor, 3D, N = 3: one warp per zone
// ---------------------------------------------------------------------------
template <typename T> struct FactSmem {
  // per-zone layout (elements of T).  w at the spatial nodes: every stage that
  // reads it is lane-static in the node (s = lane, lane + 32), so FP64 keeps
  // it in registers (its shared memory sets its occupancy); FP32 keeps it here
  // (its registers set its occupancy)
  static constexpr bool WN_REG = sizeof(T) == 8;
  static constexpr int W = 0;                          // w[5][20]
  static constexpr int WN = W + 100;                   // wn[5][64] (FP32)
  static constexpr int G = WN + (WN_REG ? 0 : 320);    // g[5][15]
  static constexpr int R1 = WN_REG ? G + 75 : G + 76;  // (FP32: 16-byte aligned C rows)
  static constexpr int R2 = R1 + 960;                  // A/B, Y1 (1728), Y3
  static constexpr int SIZE = R2 + 1728;               // 2863 (FP64), 3184 (FP32)
};

// the mass-row source table, copied to shared memory once per block
// (lane-divergent reads of constant memory are serialised; shared memory is
// not).  The other enumerations are compile-time functions or packed
// constants (p3idx, tri2idx, gmidx, kTri2P, ...).
struct FactIdx {
  // sources of the mass row of G (mass_gmode), per direction d and G-mode b:
  // [0] w, [1..3] g with e = 0..2 of the momentum mode one degree up in d
  // (offsets into the w / g rows, 255 = none), [4] w of the mode three degrees
  // up (b = 0 only), [5] the derivative factor of the first (1, 2 or 3)
  uint8_t mass_src[3][6][16];
};
__constant__ FactIdx c_fidx;

template <typename T>
__device__ __forceinline__ bool state_physical5(const T* u, T gm1) {
  return state_physical<3, T>(u, gm1);
}

// Lane mappings of the factorised kernel.  The contraction stages of w at the
// nodes (T1, T2) and of the G evaluation (E1-E3) use static mappings: each
// lane owns fixed indices and the rest are compile-time loops with
// constant-bank basis operands; some lanes idle, but every lane runs the same
// trip counts.  The two projection steps choose per precision: static in FP32
// (issue-bound: fewer loads and address computations), strided item loops over
// all 32 lanes in FP64 (fixed four-term sums, so no lane waits; the DP pipe is
// charged per warp instruction whatever the active lane count).
enum : unsigned { kStP1 = 1, kStP2 = 2 };
template <typename T> constexpr unsigned kStatic = sizeof(T) == 4 ? (kStP1 | kStP2) : 0u;

// compile-time enumerations: predict_index.cuh

// Mass row of the new G.  The mass flux of direction d is the momentum
// q_{1+d} = w_{1+d} - sum_g g_{1+d} P_a P_b P_c I_e(tau): a polynomial of total
// degree <= 3 in (x, y, z, tau), the space the fluxes are projected onto.  The
// Gauss rules of the projection (4 points per axis) integrate its products with
// the test functions exactly, so the projection is the polynomial itself and
// its derivative follows from the coefficients: I_0 = (L_0 + L_1)/2,
// I_e = (L_{e+1} - L_{e-1}) / (2(2e+1)), dP1 = P0, dP2 = 2 P1, dP3 = 3 P2 + P0/10.
// Same value as projecting the node fluxes, up to rounding, without the node
// work.  Branch-free over a source table (FactIdx::mass_src), so lanes with
// different G-modes do not diverge.  Reads the previous G (rows 1..3) and w.
// One direction's term, lamd * d/dx_d of the momentum q_{1+d}, of G-mode b
// (0 for the unused column b = 15).  The coefficient of L_e of a source mode
// is cw w + c0 g_0 + c1 g_1 + c2 g_2 with (1, -1/2, 1/6, 0), (0, -1/2, 0, 1/10),
// (0, 0, -1/6, 0) for e = 0, 1, 2.
template <typename T>
__device__ __forceinline__ T mass_gmode_dir(const T* z, const FactIdx& ix, int b, int d, T lamd) {
  const int e = unpack(kGmE, 2, b);
  const T* zw = z + FactSmem<T>::W;
  const T* zg = z + FactSmem<T>::G;
  const int ow = ix.mass_src[d][0][b], o0 = ix.mass_src[d][1][b], o1 = ix.mass_src[d][2][b];
  const int o2 = ix.mass_src[d][3][b], o3 = ix.mass_src[d][4][b];
  const T w = ow != 255 ? zw[ow] : T(0);
  const T g0 = o0 != 255 ? zg[o0] : T(0);
  const T g1 = o1 != 255 ? zg[o1] : T(0);
  const T g2 = o2 != 255 ? zg[o2] : T(0);
  const T w3 = o3 != 255 ? zw[o3] : T(0);
  const T cw = e == 0 ? T(1) : T(0);
  const T c0 = e == 2 ? T(0) : T(-0.5);
  const T c1 = e == 0 ? T(1.0 / 6.0) : e == 2 ? T(-1.0 / 6.0) : T(0);
  const T c2 = e == 1 ? T(0.1) : T(0);
  const T m = fma(c2, g2, fma(c1, g1, fma(c0, g0, cw * w)));
  return lamd * fma(T(ix.mass_src[d][5][b]), m, T(0.1) * w3);
}
// Mass row of G-mode (lane & 15): lanes 0-15 take directions 0 and 1, lanes
// 16-31 direction 2, combined by one shuffle (valid in lanes < 15).  Every
// lane runs the same instructions: a masked lane would cost its DP slot.
template <typename T>
__device__ __forceinline__ T mass_gmode(const T* z, const FactIdx& ix, int lane, const T lam[3]) {
  const int b = lane & 15;
  const bool lo = lane < 16;
  const T p0 = mass_gmode_dir<T>(z, ix, b, lo ? 0 : 2, lo ? lam[0] : lam[2]);
  const T p1 = mass_gmode_dir<T>(z, ix, b, lo ? 1 : 2, lo ? lam[1] : lam[2]);
  T part = lo ? p0 + p1 : p0;
  part += __shfl_down_sync(0xffffffffu, part, 16);
  return part;
}

// Picard projection of the node fluxes of the momentum and energy rows (the
// mass row by mass_gmode).  Y1 holds the 9 distinct flux entries ("row sets")
// r at the nodes: 0..2 the diagonal momentum flux of direction r, 3..5 the
// off-diagonal momentum flux rho v_a v_b of the pairs (0,1), (0,2), (1,2),
// 6..8 the energy flux of direction r - 6.  Direction d's flux of the variable
// 1 + v' (v' = 0..3) is projected with the plain basis along the two axes
// other than d (P1, P2) and with the derivative factors along d (P3).  P1 takes
// the axis c1(r) first: for an off-diagonal entry the axis that is neither of
// its two directions, so that one P1 serves both; P2 then contracts the
// remaining axis c2 of each (d, v'), and Y3 keeps the canonical order of the
// two transverse modes (lower axis first).
template <typename T, int EMAX>
__device__ __forceinline__ void fact_project(T* z, const Tabs<T>& tb, const FactIdx& ix, int lane,
                                             const T lam[3]) {
  constexpr int NPE = EMAX == 0 ? 3 : 6;     // (p,e) pairs with e <= EMAX
  constexpr int NTR = EMAX == 0 ? 6 : 10;    // (p,q,e) triples with e <= EMAX
  constexpr int NGE = EMAX == 0 ? 10 : 15;   // G-modes with e <= EMAX
  const T* Y1 = z + FactSmem<T>::R2;         // [r][s][e3]          (e3 stride 3)
  T* Y2 = z + FactSmem<T>::R1;               // [r][n2][pe]         (pe stride 6)
  T* Y3 = z + FactSmem<T>::R2;               // [d][v'][n1][tri]    (tri stride 10; Y1 is dead)
  // the mass row from the previous G, before P3 overwrites it
  const T gmass = mass_gmode<T>(z, ix, lane, lam);   // all lanes take part (shuffle)
  // Static lane mappings (kStatic): P1 lanes own (n2, a group of row sets),
  // P2 lanes own (n1, d, v'); the remaining indices are compile-time loops, so
  // the basis values are uniform constant-bank operands.
  const Tabs<T>& tc = tabs<T>(3);
  if constexpr ((kStatic<T> & kStP1) != 0) {
    // lanes own (n2, row sets 0-4 or 5-8) and compute every (p,e) pair of a
    // row set from its 4 x (EMAX+1) values, loaded once
    const int n2 = lane & 15, vh = lane >> 4;
    const int a0 = n2 & 3, a1 = n2 >> 2;
#pragma unroll 1
    for (int r = vh ? 5 : 0; r < (vh ? 9 : 5); ++r) {
      const int c1 = unpack(kP1C1, 4, r);
      const int str = 3 << (2 * c1);
      const int base = c1 == 0 ? 4 * a0 + 16 * a1 : c1 == 1 ? a0 + 16 * a1 : a0 + 4 * a1;
      const T* yv = Y1 + (r * 64 + base) * 3;
      T y[EMAX + 1][4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e <= EMAX; ++e) y[e][m] = yv[m * str + e];
#pragma unroll
      for (int pe = 0; pe < NPE; ++pe) {
        const int p = pair2_p(pe), e = pair2_e(pe);
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) acc = fma(y[e][m], tc.WPN[p][m], acc);
        Y2[(r * 16 + n2) * 6 + pe] = acc;
      }
    }
  } else {
#pragma unroll 2
    for (int it = lane; it < 9 * 16 * NPE; it += 32) {
      const int pe = it % NPE, rest = it / NPE, n2 = rest % 16, r = rest / 16;
      const int p = pair2_p(pe), e = pair2_e(pe);
      const int c1 = unpack(kP1C1, 4, r);
      const int a0 = n2 & 3, a1 = n2 >> 2;
      const int str = 3 << (2 * c1);
      const int base = c1 == 0 ? 4 * a0 + 16 * a1 : c1 == 1 ? a0 + 16 * a1 : a0 + 4 * a1;
      const T* yv = Y1 + (r * 64 + base) * 3 + e;
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) acc = fma(yv[m * str], tb.WPN[p][m], acc);
      Y2[(r * 16 + n2) * 6 + pe] = acc;
    }
  }
  __syncwarp();
  if constexpr ((kStatic<T> & kStP2) != 0) {
    // lanes own (n1, d, v'): 48 items in two rounds
#pragma unroll 1
    for (int it = lane; it < 48; it += 32) {
      const int n1 = it & 3, dv = it >> 2;
      const int r = unpack(kP2Row, 4, dv);
      const bool lo = unpack(kP2Lo, 4, dv) != 0, swap = unpack(kP2Swap, 4, dv) != 0;
      const int nbase = lo ? n1 : 4 * n1, nstr = lo ? 4 : 1;
      const T* y2 = Y2 + r * 16 * 6;
      T y[NPE][4];  // every operand once
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int pe = 0; pe < NPE; ++pe) y[pe][m] = y2[(nbase + m * nstr) * 6 + pe];
#pragma unroll
      for (int pe = 0; pe < NPE; ++pe) {
        const int qq = pair2_p(pe), e = pair2_e(pe);
#pragma unroll
        for (int p = 0; p <= 2 - qq - e; ++p) {
          T acc = T(0);
#pragma unroll
          for (int m = 0; m < 4; ++m) acc = fma(y[pe][m], tc.WPN[p][m], acc);
          Y3[(dv * 4 + n1) * 10 + (swap ? tri2idx(qq, p, e) : tri2idx(p, qq, e))] = acc;
        }
      }
    }
  } else {
#pragma unroll 2
    for (int it = lane; it < 12 * 4 * NTR; it += 32) {
      // tr = (p, qq, e): p the mode along c2 (this step), qq along c1 (P1)
      const int tr = it % NTR, rest = it / NTR, n1 = rest % 4, dv = rest / 4;
      const int p = unpack(kTri2P, 2, tr), qq = unpack(kTri2Q, 2, tr), e = unpack(kTri2R, 2, tr);
      const int r = unpack(kP2Row, 4, dv);
      const int pe = p2idx(qq, e);
      const bool lo = unpack(kP2Lo, 4, dv) != 0;
      const T* y2 = Y2 + r * 16 * 6 + pe;
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) acc = fma(y2[(lo ? n1 + 4 * m : m + 4 * n1) * 6], tb.WPN[p][m], acc);
      Y3[(dv * 4 + n1) * 10 + (unpack(kP2Swap, 4, dv) ? tri2_fast(qq, p, e) : tr)] = acc;
    }
  }
  __syncwarp();
  // P3: contract the derivative dimension with the Q factors, sum over d
  for (int it = lane; it < 4 * NGE; it += 32) {
    int b = it % NGE;
    int v = it / NGE;
    const int a = unpack(kGmA, 2, b), bb = unpack(kGmB, 2, b), c = unpack(kGmC, 2, b), e = unpack(kGmE, 2, b);
    int slack = 3 - (a + bb + c + e);
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const int t0 = tri2_fast(bb, c, e), t1 = tri2_fast(a, c, e), t2 = tri2_fast(a, bb, e);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      s0 = fma(Y3[((0 * 4 + v) * 4 + m) * 10 + t0], tb.QN[a][slack][m], s0);
      s1 = fma(Y3[((1 * 4 + v) * 4 + m) * 10 + t1], tb.QN[bb][slack][m], s1);
      s2 = fma(Y3[((2 * 4 + v) * 4 + m) * 10 + t2], tb.QN[c][slack][m], s2);
    }
    z[FactSmem<T>::G + (v + 1) * 15 + b] = fma(lam[0], s0, fma(lam[1], s1, lam[2] * s2));
  }
  if (lane < NGE) z[FactSmem<T>::G + lane] = gmass;
  if (EMAX == 0) {
    for (int it = lane; it < 5 * 5; it += 32) z[FactSmem<T>::G + (it / 5) * 15 + 10 + it % 5] = T(0);
  }
  __syncwarp();
}

// Node stage of the Picard sweeps (factorised kernel): the fluxes of the
// 4 time points of a node, time-contracted onto e = 0..2.  The time nodes are
// taken in symmetric pairs (t, 3 - t): with w_{3-t} = w_t and L_e(1 - tau) =
// (-1)^e L_e(tau), the even modes take the sum of the pair's fluxes and the
// odd mode their difference.  The momentum flux rho v_d v_e is symmetric in
// (d, e), so its three off-diagonal entries are formed and contracted once;
// the mass fluxes are not needed (mass_gmode): 9 entries per state,
// f = diagonal[3], off-diagonal[3] (01, 02, 12), energy[3].
template <typename T> struct NodeAcc {
  T a[9][3];
};

template <typename T>
__device__ __forceinline__ void sym_fluxes(const T* qn, T irho, T gm1, T* f) {
  T vel[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) vel[d] = qn[1 + d] * irho;
  T m2 = qn[1] * vel[0];
  m2 = fma(qn[2], vel[1], m2);
  m2 = fma(qn[3], vel[2], m2);
  const T p = gm1 * (qn[4] - T(0.5) * m2);
  const T Ep = qn[4] + p;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f[d] = fma(qn[1 + d], vel[d], p);
    f[6 + d] = Ep * vel[d];
  }
  f[3] = qn[1] * vel[1];
  f[4] = qn[1] * vel[2];
  f[5] = qn[2] * vel[2];
}

template <typename T>
__device__ __forceinline__ void accumulate_pair(NodeAcc<T>& acc, const T* fa, const T* fb,
                                                const Tabs<T>& tc, int tp) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const T sum = fa[k] + fb[k], dif = fa[k] - fb[k];
    acc.a[k][0] = fma(tc.WLT[0][tp], sum, acc.a[k][0]);
    acc.a[k][1] = fma(tc.WLT[1][tp], dif, acc.a[k][1]);
    acc.a[k][2] = fma(tc.WLT[2][tp], sum, acc.a[k][2]);
  }
}

// Y1[r][s][e]: the 9 distinct entries in NodeAcc order (fact_project)
template <typename T>
__device__ __forceinline__ void store_node_y1(T* Y1, int s, const NodeAcc<T>& acc) {
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int e = 0; e < 3; ++e) Y1[(r * 64 + s) * 3 + e] = acc.a[r][e];
}

// Face states of one zone (whole warp): the time integral of G at the two face
// time points (shared by all directions), then per (direction, side, variable)
// the normal axis at +-1/2 and the two transverse axes at the face Gauss
// points, the positivity fallback and the store.  sg holds G with rows GS
// entries apart; scratch takes 340 entries.
// Time integral of G at the two face time points (shared by all directions
// of a zone): gt[v][it][tri], 100 entries, over `nl` lanes from lane l0.
template <typename T, int GS>
__device__ __forceinline__ void face_gt(const T* sg, T* gt, const Tabs<T>& tb, int l0, int nl) {
  for (int it = l0; it < 100; it += nl) {
    int tr = it % 10, rest = it / 10, tq = rest % 2, v = rest / 2;
    const int a = unpack(kTri2P, 2, tr), b = unpack(kTri2Q, 2, tr), c = unpack(kTri2R, 2, tr);
    T acc = T(0);
    for (int e = 0; e <= 2 - a - b - c; ++e) acc = fma(sg[v * GS + gm_fast(a, b, c, e)], tb.ITF[e][tq], acc);
    gt[it] = acc;
  }
}

// Face values of one (variable v, direction-side ds) combination: the normal
// axis at +-1/2, then the two transverse axes at the face Gauss points, for the
// w part and, per face time point, the G part.  fv[(ds*8 + q)*5 + v], q = i1 +
// 2*(i2 + 2*it), as the probes document.
template <typename T>
__device__ __forceinline__ void face_values_reg(const T* sw, const T* gt, const Tabs<T>& tb, int v, int ds,
                                                T (&out)[8]) {
  const int d = ds >> 1, side = ds & 1;
  // axes: n = d (normal), t1 < t2 the transverse ones.  Every loop below
  // is unrolled over compile-time exponents; the mode index of (an on the
  // normal axis, p1 on t1, p2 on t2) is one of three constants, picked by d
  // w part: contract the normal axis at the face, then t1, then t2
  T wn2[10];  // (p1, p2) with p1 + p2 <= 3, index p3idx(p1, p2)
#pragma unroll
  for (int p2 = 0; p2 <= 3; ++p2)
#pragma unroll
    for (int p1 = 0; p1 <= 3 - p2; ++p1) {
      T acc = T(0);
#pragma unroll
      for (int an = 0; an <= 3 - p1 - p2; ++an) {
        const int m = d == 0 ? simplex_idx(3, an, p1, p2) : d == 1 ? simplex_idx(3, p1, an, p2)
                                                                  : simplex_idx(3, p1, p2, an);
        acc = fma(sw[v * 20 + m], tb.PE[an][side], acc);
      }
      wn2[p3idx(p1, p2)] = acc;
    }
  T w3[2][4];  // [i1][p2]
#pragma unroll
  for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
    for (int p2 = 0; p2 < 4; ++p2) {
      T acc = T(0);
#pragma unroll
      for (int p1 = 0; p1 <= 3 - p2; ++p1) acc = fma(wn2[p3idx(p1, p2)], tb.PF[p1][i1], acc);
      w3[i1][p2] = acc;
    }
  // G part per face time point
  T gv[2][2][2];  // [it][i1][i2]
#pragma unroll
  for (int tq = 0; tq < 2; ++tq) {
    const T* gtv = gt + (v * 2 + tq) * 10;
    T gn2[6];  // (p1, p2) with p1 + p2 <= 2, index p2idx(p1, p2)
#pragma unroll
    for (int p2 = 0; p2 <= 2; ++p2)
#pragma unroll
      for (int p1 = 0; p1 <= 2 - p2; ++p1) {
        T acc = T(0);
#pragma unroll
        for (int an = 0; an <= 2 - p1 - p2; ++an) {
          const int m = d == 0 ? tri2idx(an, p1, p2) : d == 1 ? tri2idx(p1, an, p2) : tri2idx(p1, p2, an);
          acc = fma(gtv[m], tb.PE[an][side], acc);
        }
        gn2[p2idx(p1, p2)] = acc;
      }
#pragma unroll
    for (int i1 = 0; i1 < 2; ++i1) {
      T g3[3];
#pragma unroll
      for (int p2 = 0; p2 < 3; ++p2) {
        T acc = T(0);
#pragma unroll
        for (int p1 = 0; p1 <= 2 - p2; ++p1) acc = fma(gn2[p2idx(p1, p2)], tb.PF[p1][i1], acc);
        g3[p2] = acc;
      }
#pragma unroll
      for (int i2 = 0; i2 < 2; ++i2) {
        T acc = T(0);
#pragma unroll
        for (int p2 = 0; p2 < 3; ++p2) acc = fma(g3[p2], tb.PF[p2][i2], acc);
        gv[tq][i1][i2] = acc;
      }
    }
  }
#pragma unroll
  for (int i1 = 0; i1 < 2; ++i1)
#pragma unroll
    for (int i2 = 0; i2 < 2; ++i2) {
      T acc = T(0);
#pragma unroll
      for (int p2 = 0; p2 < 4; ++p2) acc = fma(w3[i1][p2], tb.PF[p2][i2], acc);
#pragma unroll
      for (int tq = 0; tq < 2; ++tq) out[i1 + 2 * (i2 + 2 * tq)] = acc - gv[tq][i1][i2];
    }
}
// stores fv[(ds*8 + q)*5 + v], q = i1 + 2*(i2 + 2*it), as the probes document
template <typename T>
__device__ __forceinline__ void face_values_store(T* fv, int v, int ds, const T (&out)[8]) {
#pragma unroll
  for (int qq = 0; qq < 8; ++qq) fv[(ds * 8 + qq) * 5 + v] = out[qq];
}
template <typename T>
__device__ __forceinline__ void face_values_one(const T* sw, const T* gt, T* fv, const Tabs<T>& tb, int v, int ds) {
  T out[8];
  face_values_reg<T>(sw, gt, tb, v, ds, out);
  face_values_store<T>(fv, v, ds, out);
}

// face_gt for one zone on 16 lanes: lanes l < 10 own (v, it) = (l >> 1, l & 1)
// and every triple with compile-time indices
template <typename T, int GS>
__device__ __forceinline__ void face_gt_vt(const T* sg, T* gt, const Tabs<T>& tb, int l) {
  if (l < 10) {
    const int v = l >> 1, tq = l & 1;
    T itf[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) itf[e] = tb.ITF[e][tq];
    const T* g = sg + v * GS;
    T* o = gt + (v * 2 + tq) * 10;
#pragma unroll
    for (int tr = 0; tr < 10; ++tr) {
      const int a = tri2_p(tr), b = tri2_q(tr), c = tri2_r(tr);
      T acc = T(0);
#pragma unroll
      for (int e = 0; e <= 2 - a - b - c; ++e) acc = fma(g[gmidx(a, b, c, e)], itf[e], acc);
      o[tr] = acc;
    }
  }
}

template <typename T, int GS>
__device__ __forceinline__ void fact_face_states(const Geo& q, const T* sw, const T* sg, T* scratch,
                                                 const Tabs<T>& tb, int lane, T gm1, long long nb, long long r,
                                                 T* __restrict__ FS) {
  // face states into shared memory.  Factorised evaluation: the time
  // integral of G at the two face time points (shared by all directions),
  // then per (direction, side, variable) the normal axis at +-1/2 and the two
  // transverse axes at the face Gauss points.  Row = (d*2+side)*8 + q with
  // q = i1 + 2*(i2 + 2*it), as the probes document.
  T* fv = scratch;                      // [48][5] face values
  T* gt = fv + 240;                     // [v][it][tri] time-integrated G, 100
  face_gt<T, GS>(sg, gt, tb, lane, 32);
  __syncwarp();
  if (lane < 30) face_values_one<T>(sw, gt, fv, tb, lane % 5, lane / 5);
  __syncwarp();
  bool bad = false;
  if (q.fallback)
    for (int row = lane; row < 48; row += 32) bad = bad || !state_physical5<T>(fv + row * 5, gm1);
  bad = __any_sync(0xffffffffu, bad) && q.fallback;
  if (bad && lane == 0 && q.fb_count) atomicAdd(q.fb_count, 1ULL);
  __syncwarp();
  for (int it = lane; it < 240; it += 32) {
    int v = it % 5, row = it / 5;
    FS[((long long)row * 5 + v) * nb + r] = bad ? sw[v * 20] : fv[row * 5 + v];
  }
}

// Register budgets: FP32 at 8 blocks of two zone-warps per SM (its shared
// memory allows 8); FP64 at most ~170 registers (its shared memory allows 4
// blocks; more registers measured slower)
template <typename T, int WPB>
__global__ void __launch_bounds__(32 * WPB, sizeof(T) == 4 ? 8 : 6) k_predict_fact(Geo q, Region box, const T* __restrict__ W,
                                                           const double* __restrict__ d_dt, int picard,
                                                           const T* __restrict__ tab, PTabLayout L,
                                                           T* __restrict__ FS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tabs<T>& tb = *reinterpret_cast<Tabs<T>*>(smem_raw);
  FactIdx& ix = *reinterpret_cast<FactIdx*>(smem_raw + ((sizeof(Tabs<T>) + 15) / 16) * 16);
  T* smem = reinterpret_cast<T*>(smem_raw + ((sizeof(Tabs<T>) + 15) / 16) * 16 + ((sizeof(FactIdx) + 15) / 16) * 16);
  {
    const int* src = reinterpret_cast<const int*>(&tabs<T>(3));
    int* dst = reinterpret_cast<int*>(&tb);
    for (int i = threadIdx.x; i < (int)(sizeof(Tabs<T>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    const int8_t* s8 = reinterpret_cast<const int8_t*>(&c_fidx);
    int8_t* d8 = reinterpret_cast<int8_t*>(&ix);
    for (int i = threadIdx.x; i < (int)sizeof(FactIdx); i += blockDim.x) d8[i] = s8[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  T* z = smem + wib * FactSmem<T>::SIZE;
  const long long nb = box.size();
  const double dt = *d_dt;
  T lam[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) lam[d] = (T)(dt / q.dx[d]);
  const T gm1 = (T)(q.gamma - 1.0);
  const T* FW = tab + L.fw;
  const T* FG = tab + L.fg;
  for (long long r = (long long)blockIdx.x * WPB + wib; r < nb; r += (long long)gridDim.x * WPB) {
    T* sw = z + FactSmem<T>::W;
    T* swn = z + FactSmem<T>::WN;          // FP32
    T wnr[2][5];                            // FP64: w at the nodes s = lane, lane + 32
    T* sg = z + FactSmem<T>::G;
    for (int it = lane; it < 100; it += 32) sw[it] = W[(long long)it * nb + r];
    __syncwarp();
    // w at the 64 spatial nodes: contract a, then b, then c
    {
      T* T1 = z + FactSmem<T>::R1;        // [v][i][pair3]   200
      T* T2 = T1 + 200;                   // [v][i][j][c]    320
      {
        // T1[v][i][(b,c)]: lanes own (i, v), compile-time (b, c, a)
        if (lane < 20) {
          const int i = lane & 3, v = lane >> 2;
          T pni[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) pni[a] = tb.PN[a][i];
#pragma unroll
          for (int c = 0; c <= 3; ++c)
#pragma unroll
            for (int b = 0; b <= 3 - c; ++b) {
              T acc = T(0);
#pragma unroll
              for (int a = 0; a <= 3 - b - c; ++a) acc = fma(sw[v * 20 + simplex_idx(3, a, b, c)], pni[a], acc);
              T1[(v * 4 + i) * 10 + p3idx(b, c)] = acc;
            }
        }
      }
      __syncwarp();
      {
        {
          // T2[v][i][j][c]: lanes own (i, j) and half of the variables
          const int i = lane & 3, j = (lane >> 2) & 3, h = lane >> 4;
          T pnj[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) pnj[b] = tb.PN[b][j];
#pragma unroll 1
          for (int v = h; v < 5; v += 2) {
            const T* t1 = T1 + (v * 4 + i) * 10;
            T* t2 = T2 + ((v * 4 + i) * 4 + j) * 4;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              T acc = T(0);
#pragma unroll
              for (int b = 0; b <= 3 - c; ++b) acc = fma(t1[p3idx(b, c)], pnj[b], acc);
              t2[c] = acc;
            }
          }
        }
        __syncwarp();
        // w at the spatial nodes: lanes own the nodes s = lane and lane + 32
#pragma unroll
        for (int hs = 0; hs < 2; ++hs) {
          const int s = lane + 32 * hs;
          const int i = s & 3, j = (s >> 2) & 3, k = s >> 4;
          T pnk[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) pnk[c] = tb.PN[c][k];
          if constexpr (FactSmem<T>::WN_REG) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const T* t2 = T2 + ((v * 4 + i) * 4 + j) * 4;
              T acc = T(0);
#pragma unroll
              for (int c = 0; c < 4; ++c) acc = fma(t2[c], pnk[c], acc);
              wnr[hs][v] = acc;
            }
          } else {
#pragma unroll 1
            for (int v = 0; v < 5; ++v) {
              const T* t2 = T2 + ((v * 4 + i) * 4 + j) * 4;
              T acc = T(0);
#pragma unroll
              for (int c = 0; c < 4; ++c) acc = fma(t2[c], pnk[c], acc);
              swn[v * 64 + s] = acc;
            }
          }
        }
      }
      __syncwarp();
    }
    for (int it = lane; it < 75; it += 32) sg[it] = T(0);
    __syncwarp();
    T* Y1 = z + FactSmem<T>::R2;
    if (picard >= 1) {
      // sweep 0: flux at the spatial nodes, time-independent
#pragma unroll
      for (int hs = 0; hs < 2; ++hs) {
        const int s = lane + 32 * hs;
        T qn[5], F[3][5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = FactSmem<T>::WN_REG ? wnr[hs][v] : swn[v * 64 + s];
        phys_fluxes<3, T>(qn, gm1, F);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          Y1[(d * 64 + s) * 3] = F[d][1 + d];          // diagonal momentum
          Y1[((6 + d) * 64 + s) * 3] = F[d][4];        // energy
        }
        Y1[(3 * 64 + s) * 3] = F[0][2];                // rho v_x v_y
        Y1[(4 * 64 + s) * 3] = F[0][3];                // rho v_x v_z
        Y1[(5 * 64 + s) * 3] = F[1][3];                // rho v_y v_z
      }
      __syncwarp();
      fact_project<T, 0>(z, tb, ix, lane, lam);
    }
    for (int sweep = 1; sweep < picard; ++sweep) {
      T* A = z + FactSmem<T>::R2;   // [v][tri][t]        200 (dead before Y1 is written)
      T* B = A + 200;               // [v][i][pair2][t]   480 (dead before Y1 is written)
      T* C = z + FactSmem<T>::R1;   // [v][i][j][c][t]    960
      // E1: A[v][(a,b,c)][t] = sum_e g[(a,b,c,e)] I_e(tau_t); lanes own (t, v)
      {
        if (lane < 20) {
          const int t = lane & 3, v = lane >> 2;
          T it_[3];
#pragma unroll
          for (int e = 0; e < 3; ++e) it_[e] = tb.IT[e][t];
#pragma unroll
          for (int tr = 0; tr < 10; ++tr) {
            const int a = tri2_p(tr), b = tri2_q(tr), c = tri2_r(tr);
            T acc = T(0);
#pragma unroll
            for (int e = 0; e <= 2 - a - b - c; ++e) acc = fma(sg[v * 15 + gmidx(a, b, c, e)], it_[e], acc);
            A[(v * 10 + tr) * 4 + t] = acc;
          }
        }
      }
      __syncwarp();
      // E2: B[v][i][(b,c)][t] = sum_a A[(a,b,c)][t] P_a(x_i); lanes own (i, t, half of v)
      {
        {
          const int i = lane & 3, t = (lane >> 2) & 3, h = lane >> 4;
          T pni[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) pni[a] = tb.PN[a][i];
#pragma unroll 1
          for (int v = h; v < 5; v += 2) {
#pragma unroll
            for (int pc = 0; pc < 6; ++pc) {
              const int b = pair2_p(pc), c = pair2_e(pc);
              T acc = T(0);
#pragma unroll
              for (int a = 0; a <= 2 - b - c; ++a) acc = fma(A[(v * 10 + tri2idx(a, b, c)) * 4 + t], pni[a], acc);
              B[((v * 4 + i) * 6 + pc) * 4 + t] = acc;
            }
          }
        }
      }
      __syncwarp();
      // E3: C[v][i][j][c][t] = sum_b B[i][(b,c)][t] P_b(y_j); lanes own (i, j, parity of t)
      {
        {
          const int i = lane & 3, j = (lane >> 2) & 3, h = lane >> 4;
          T pnj[3];
#pragma unroll
          for (int b = 0; b < 3; ++b) pnj[b] = tb.PN[b][j];
#pragma unroll 1
          for (int v = 0; v < 5; ++v) {
#pragma unroll
            for (int tt = 0; tt < 2; ++tt) {
              const int t = h + 2 * tt;
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                T acc = T(0);
#pragma unroll
                for (int b = 0; b <= 2 - c; ++b) acc = fma(B[((v * 4 + i) * 6 + p2idx(b, c)) * 4 + t], pnj[b], acc);
                C[((((v * 4 + i) * 4 + j) * 3 + c) * 4) + t] = acc;
              }
            }
          }
        }
      }
      __syncwarp();
      // nodes: q = wn - sum_c C P_c(z_k); fluxes; time contraction into Y1
      // (the time weights have compile-time indices: constant-bank operands)
      const Tabs<T>& tc = tabs<T>(3);
      if constexpr (sizeof(T) == 4) {
        // FP32: each C row (the 4 time points of one (v, i, j, c)) as one
        // 16-byte shared-memory load
        for (int s = lane; s < 64; s += 32) {
          const int i = s & 3, j = (s >> 2) & 3, k = s >> 4;
          T pnk[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) pnk[c] = tb.PN[c][k];
          float4 cv[5][3];
#pragma unroll
          for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              cv[v][c] = *reinterpret_cast<const float4*>(C + (((v * 4 + i) * 4 + j) * 3 + c) * 4);
          NodeAcc<T> acc = {};
#pragma unroll
          for (int tp = 0; tp < 2; ++tp) {
            T f[2][9], qn[2][5];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int t = h ? 3 - tp : tp;
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                T x = swn[v * 64 + s];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  const float4 q4 = cv[v][c];
                  const T cc = t == 0 ? q4.x : t == 1 ? q4.y : t == 2 ? q4.z : q4.w;
                  x = fma(-cc, pnk[c], x);
                }
                qn[h][v] = x;
              }
            }
            T ia, ib;
            recip_pair<T>(qn[0][0], qn[1][0], ia, ib);
            sym_fluxes<T>(qn[0], ia, gm1, f[0]);
            sym_fluxes<T>(qn[1], ib, gm1, f[1]);
            accumulate_pair<T>(acc, f[0], f[1], tc, tp);
          }
          store_node_y1<T>(Y1, s, acc);
        }
      } else
#pragma unroll 1
      for (int hs = 0; hs < 2; ++hs) {
        const int s = lane + 32 * hs;
        int i = s & 3, j = (s >> 2) & 3, k = s >> 4;
        T pnk[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) pnk[c] = tb.PN[c][k];
        NodeAcc<T> acc = {};
#pragma unroll
        for (int tp = 0; tp < 2; ++tp) {
          T f[2][9], qn[2][5];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int t = h ? 3 - tp : tp;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              T x = FactSmem<T>::WN_REG ? (hs ? wnr[1][v] : wnr[0][v]) : swn[v * 64 + s];
#pragma unroll
              for (int c = 0; c < 3; ++c) x = fma(-C[((((v * 4 + i) * 4 + j) * 3 + c) * 4) + t], pnk[c], x);
              qn[h][v] = x;
            }
          }
          T ia, ib;
          recip_pair<T>(qn[0][0], qn[1][0], ia, ib);
          sym_fluxes<T>(qn[0], ia, gm1, f[0]);
          sym_fluxes<T>(qn[1], ib, gm1, f[1]);
          accumulate_pair<T>(acc, f[0], f[1], tc, tp);
        }
        store_node_y1<T>(Y1, s, acc);
      }
      __syncwarp();
      fact_project<T, 2>(z, tb, ix, lane, lam);
    }
    fact_face_states<T, 15>(q, sw, sg, z + FactSmem<T>::R1, tb, lane, gm1, nb, r, FS);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// FP32 predictor, 3D, N = 3, with node lines in registers
// ---------------------------------------------------------------------------
// The FP32 form of the factorised kernel above is bound by shared-memory
// bandwidth: every contraction stage reads its operands from shared memory
// for one FMA each.  Here a zone takes 16 lanes (two zones per warp) and each
// lane owns one line of four nodes along z, (x_i, y_j, z_k), k = 0..3.  The
// evaluation of the Picard iterate at the line's 16 space-time points, the
// fluxes, their time contraction and the first projection step (along z)
// happen in the lane's registers; only the z-projected fluxes go through
// shared memory to the two remaining projection steps.
//
// Row sets at the nodes (NodeAcc order): 0..2 the diagonal momentum flux of
// direction r, 3..5 the off-diagonal rho v_a v_b of (0,1), (0,2), (1,2), 6..8
// the energy flux of direction r - 6.  The z step keeps, per row, the pairs
// (p, e) of z-mode and time mode in nine slots with the same positions in
// every row:
//   slot  0     1     2     3     4     5     6     7     8
//   (p,e) (1,0) (1,1) (2,0) (0,0) (0,1) (0,2) (3,0) (2,1) (1,2)
// Slots 0-5 (p + e <= 2) serve the directions x and y, for which z is a plain
// axis; slots 0-2 and 6-8 (p >= 1, p + e <= 3) serve direction z, whose
// derivative is applied to the projection coefficients afterwards
// (dP1 = P0, dP2 = 2 P1, dP3 = 3 P2 + P0/10).  The second step contracts one
// plain axis in three rounds, each for the four variables 1..4:
//   round 0: direction x, contract y over slots 0-5  (rows 0, 3, 4, 6)
//   round 1: direction y, contract x over slots 0-5  (rows 3, 1, 5, 7)
//   round 2: direction z, contract y over slots 0-2, 6-8 (rows 4, 5, 2, 8)
// and the last step contracts the remaining axis: with the derivative
// factors QN in rounds 0 and 1 (the same operator as the factorised kernel),
// with the plain basis followed by the modal derivative in round 2.
__host__ __device__ constexpr int ln_p(int s) {
  return s == 0 || s == 1 || s == 8 ? 1 : s == 2 || s == 7 ? 2 : s == 6 ? 3 : 0;
}
__host__ __device__ constexpr int ln_e(int s) { return s == 1 || s == 4 || s == 7 ? 1 : s == 5 || s == 8 ? 2 : 0; }
__host__ __device__ constexpr bool ln_row_xy(int r) { return r != 2 && r != 8; }            // serves x or y
__host__ __device__ constexpr bool ln_row_z(int r) { return r == 2 || r == 4 || r == 5 || r == 8; }  // serves z
__host__ __device__ constexpr bool ln_used(int r, int s) { return s < 3 || (s < 6 ? ln_row_xy(r) : ln_row_z(r)); }
// the slots of round R (index u = 0..5)
__host__ __device__ constexpr int ln_round_slot(int R, int u) { return R == 2 && u >= 3 ? u + 3 : u; }
// largest mode of the contracted axis kept for slot s in round R (the total
// degree of the projection: <= 2 for a plain z axis, <= 3 for z's own)
__host__ __device__ constexpr int ln_qmax(int R, int s) { return (R == 2 ? 3 : 2) - ln_p(s) - ln_e(s); }
// position of (slot index u, mode q) among the 10 outputs of a round
__host__ __device__ constexpr int ln_tri(int R, int u, int q) {
  int t = 0;
  for (int uu = 0; uu < u; ++uu) t += ln_qmax(R, ln_round_slot(R, uu)) + 1;
  return t + q;
}
// row of round R for variable 1 + vv (packed: 4 bits per entry)
__host__ __device__ constexpr int ln_round_row(int R, int vv) {
  return R == 0 ? (vv == 0 ? 0 : vv == 1 ? 3 : vv == 2 ? 4 : 6)
       : R == 1 ? (vv == 0 ? 3 : vv == 1 ? 1 : vv == 2 ? 5 : 7)
                : (vv == 0 ? 4 : vv == 1 ? 5 : vv == 2 ? 2 : 8);
}
// Shared-memory base of each row of the z-projected fluxes (16 floats per
// slot): rows 160 floats apart, offset by 4 * beta(r) floats so that the four
// rows of every round start in four different groups of four banks
// (beta = 0 2 1 1 2 0 3 3 3 gives each round four distinct values).
__host__ __device__ constexpr int ln_beta(int r) {
  return r == 0 || r == 5 ? 0 : r == 2 || r == 3 ? 1 : r == 1 || r == 4 ? 2 : 3;
}
__host__ __device__ constexpr int ln_rowbase(int r) { return 160 * r + 4 * ln_beta(r); }
__host__ __device__ constexpr unsigned long long ln_pack_rowbase(int R) {
  unsigned long long k = 0;
  for (int vv = 0; vv < 4; ++vv) k |= (unsigned long long)ln_rowbase(ln_round_row(R, vv)) << (16 * vv);
  return k;
}
// per G-mode b (15 modes, gmidx order), packed 4 bits per mode: the output
// positions that the last step reads (rounds 0, 1: slot of (c, e) and the mode
// of the contracted axis; round 2: slot of (c + 1, e)) and the slack of the
// derivative factors
__host__ __device__ constexpr int ln_plain_slot(int c, int e) {   // (c, e), c + e <= 2
  return c == 1 ? (e == 0 ? 0 : 1) : c == 2 ? 2 : 3 + e;
}
__host__ __device__ constexpr int ln_z_u(int c, int e) {          // round-2 index of (c, e), c >= 1
  return c == 1 ? (e == 0 ? 0 : e == 1 ? 1 : 5) : c == 2 ? (e == 0 ? 2 : 4) : 3;
}
__host__ __device__ constexpr int ln_gm_exp(int b, int k) {
  int i = 0;
  for (int e = 0; e <= 2; ++e)
    for (int c = 0; c <= 2 - e; ++c)
      for (int bb = 0; bb <= 2 - e - c; ++bb)
        for (int a = 0; a <= 2 - e - bb - c; ++a) {
          if (i == b) return k == 0 ? a : k == 1 ? bb : k == 2 ? c : e;
          ++i;
        }
  return 0;
}
__host__ __device__ constexpr unsigned long long ln_pack_gm(int which) {
  unsigned long long k = 0;
  for (int b = 0; b < 15; ++b) {
    const int a = ln_gm_exp(b, 0), bb = ln_gm_exp(b, 1), c = ln_gm_exp(b, 2), e = ln_gm_exp(b, 3);
    int v = 0;
    if (which == 0) v = ln_tri(0, ln_plain_slot(c, e), bb);
    else if (which == 1) v = ln_tri(1, ln_plain_slot(c, e), a);
    else if (which == 2) v = ln_tri(2, ln_z_u(c + 1, e), bb);
    else v = 3 - (a + bb + c + e);
    k |= (unsigned long long)v << (4 * b);
  }
  return k;
}
constexpr unsigned long long kLnT0 = ln_pack_gm(0), kLnT1 = ln_pack_gm(1), kLnT2 = ln_pack_gm(2),
                             kLnSlack = ln_pack_gm(3);
constexpr unsigned long long kLnRB0 = ln_pack_rowbase(0), kLnRB1 = ln_pack_rowbase(1), kLnRB2 = ln_pack_rowbase(2);

// per-warp shared memory of the line kernel (floats), two zones z = 0, 1:
// w[5][20], g[5][16] (entry 15 of a row unused), the z-projected fluxes (rows
// at ln_rowbase, 1436 floats; the face stage reuses them) and the second-step
// outputs [round][vv][tri][m].  The zones' copies of the z-projected fluxes are
// 16 (mod 32) floats apart and those of the second-step outputs 4 (mod 32):
// the two zones' lanes then store to disjoint banks in both steps.
struct LineSmem {
  static constexpr int W = 0, WS = 100;
  static constexpr int G = 200, GS = 80;
  static constexpr int Y2 = 360, Y2S = 1456;
  static constexpr int Y3 = Y2 + 2 * Y2S - 16, Y3S = 484;   // 3256
  static constexpr int SIZE = Y3 + 2 * Y3S - 4;              // 4220 per warp
};

// Lane tables of the line kernel (copied to shared memory once per block).
// The mass row of G-mode b, direction d: the sources of FactIdx::mass_src
// with the g rows 16 floats apart, every offset valid (a g source that does
// not exist reads entry 15 of g row 0, which stays 0; a w source that does
// not exist reads w[0] and meets a zero factor: ms_fac where the momentum
// mode one degree up is missing, ms_c3 where the mode three degrees up is),
// and the coefficients (cw, c0, c1, c2) of the G-mode's time index; the last
// projection step's factor c + 1 of G-mode b.  No branch and no conversion
// in the kernel.
struct LineIdx {
  uint8_t ms_off[3][5][16];   // w, g0, g1, g2 (from zg), w3 (from zw)
  float ms_fac[3][16];        // 1, 2 or 3 (0: no source)
  float ms_c3[3][16];         // 0.1 or 0
  float ms_coef[16][4];       // cw, c0, c1, c2
  float lp_cfac[16];          // c + 1
};
static_assert(offsetof(LineIdx, ms_coef) % 16 == 0, "float4 rows");
__constant__ LineIdx c_lidx;
// I_e(tau_t) P_c(z_k) for (c, e) = (1, 0), (1, 1), (2, 0): [j][t][k]
__constant__ float c_ln_itpn[3][4][4];

// mass row of G-mode b, direction d (line kernel layout): as mass_gmode_dir
__device__ __forceinline__ float line_mass_dir(const float* zw, const float* zg, const LineIdx& ix, int b, int d,
                                               float lamd) {
  const float w = zw[ix.ms_off[d][0][b]];
  const float g0 = zg[ix.ms_off[d][1][b]], g1 = zg[ix.ms_off[d][2][b]], g2 = zg[ix.ms_off[d][3][b]];
  const float w3 = zw[ix.ms_off[d][4][b]];
  const float4 cf = *reinterpret_cast<const float4*>(ix.ms_coef[b]);
  const float m = fmaf(cf.w, g2, fmaf(cf.z, g1, fmaf(cf.y, g0, cf.x * w)));
  return lamd * fmaf(ix.ms_fac[d][b], m, ix.ms_c3[d][b] * w3);
}

__device__ __forceinline__ float dot4v(float4 a, float4 b) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}
__device__ __forceinline__ float dot4(float4 a, const float* bp) {
  const float4 b = *reinterpret_cast<const float4*>(bp);
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// The second and last projection steps and the mass row of the new G (the 16
// lanes of one zone; y2 holds the z-projected fluxes of the sweep).
template <int EMAX>
__device__ __forceinline__ void line_project(const float* y2, float* y3, float* sg, const float* sw,
                                             const Tabs<float>& tb, const LineIdx& ix, int l16, const float lam[3]) {
  constexpr int NGE = EMAX == 0 ? 10 : 15;
  const Tabs<float>& tc = tabs<float>(3);
  // the mass row reads the previous G: before any lane stores the new one
  float gmass = 0.f;
  if (l16 < NGE)
    gmass = line_mass_dir(sw, sg, ix, l16, 0, lam[0]) + line_mass_dir(sw, sg, ix, l16, 1, lam[1]) +
            line_mass_dir(sw, sg, ix, l16, 2, lam[2]);
  const int vv = l16 >> 2, m = l16 & 3;
  // second step, rounds 0 and 2 contract y (lanes hold i = m), round 1 x (j = m)
#pragma unroll
  for (int R = 0; R < 3; ++R) {
    const int rb = (int)((R == 0 ? kLnRB0 : R == 1 ? kLnRB1 : kLnRB2) >> (16 * vv)) & 0xffff;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int s = ln_round_slot(R, u);
      if (ln_e(s) > EMAX) continue;
      float y[4];
      if (R == 1) {
        // contiguous: one 16-byte load (row bases and slots are multiples of 4 floats)
        const float4 t4 = *reinterpret_cast<const float4*>(y2 + rb + s * 16 + 4 * m);
        y[0] = t4.x; y[1] = t4.y; y[2] = t4.z; y[3] = t4.w;
      } else {
#pragma unroll
        for (int n = 0; n < 4; ++n) y[n] = y2[rb + s * 16 + m + 4 * n];
      }
#pragma unroll
      for (int qq = 0; qq <= ln_qmax(R, s); ++qq) {
        float acc = y[0] * tc.WPN[qq][0];
#pragma unroll
        for (int n = 1; n < 4; ++n) acc = fmaf(y[n], tc.WPN[qq][n], acc);
        y3[((R * 4 + vv) * 10 + ln_tri(R, u, qq)) * 4 + m] = acc;
      }
    }
  }
  __syncwarp();
  // last step: lane l16 takes G-mode b = l16 of the four variables 1..4,
  // so that the mode's indices and its three basis rows are fetched once
  if (l16 < NGE) {
    const int b = l16;
    const int a = unpack(kGmA, 2, b), bb = unpack(kGmB, 2, b);
    const int slack = unpack(kLnSlack, 4, b);
    const float4 q0 = *reinterpret_cast<const float4*>(tb.QN[a][slack]);
    const float4 q1 = *reinterpret_cast<const float4*>(tb.QN[bb][slack]);
    const float4 pz = *reinterpret_cast<const float4*>(tb.WPN[a]);
    const float cf = ix.lp_cfac[b];
    // y3[((R * 4 + vv) * 10 + tri) * 4 + m]: variable stride 40 floats
    const float* y0 = y3 + unpack(kLnT0, 4, b) * 4;
    const float* y1 = y3 + (40 + unpack(kLnT1, 4, b)) * 4;
    const float* yz = y3 + (80 + unpack(kLnT2, 4, b)) * 4;
#pragma unroll
    for (int v4 = 0; v4 < 4; ++v4) {
      const float s0 = dot4v(*reinterpret_cast<const float4*>(y0 + 40 * v4), q0);
      const float s1 = dot4v(*reinterpret_cast<const float4*>(y1 + 40 * v4), q1);
      float s2 = cf * dot4v(*reinterpret_cast<const float4*>(yz + 40 * v4), pz);
      if (b == 0) {
        // dP3 = 3 P2 + P0/10: the z-mode 3 coefficient also feeds c = 0
        const float4 Y3z = *reinterpret_cast<const float4*>(y3 + (80 + ln_tri(2, 3, 0)) * 4 + 40 * v4);
        s2 = fmaf(0.1f, dot4(Y3z, tb.WPN[0]), s2);
      }
      sg[(v4 + 1) * 16 + b] = fmaf(lam[0], s0, fmaf(lam[1], s1, lam[2] * s2));
    }
  }
  if (l16 < NGE) sg[l16] = gmass;
  if (EMAX == 0)
    for (int it = l16; it < 25; it += 16) sg[(it / 5) * 16 + 10 + it % 5] = 0.f;
  __syncwarp();
}

// sweep-0 flux rows at one node: Z[r][s] += F_r P_p(z_k) w_k / |P_p|^2 (e = 0)
// and the time-contracted rows of the later sweeps (all used slots)
template <int EMAX>
__device__ __forceinline__ void line_z_accumulate(float (&Z)[9][9], const float (&f)[9][3], int k) {
  const Tabs<float>& tc = tabs<float>(3);
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int s = 0; s < 9; ++s)
      if (ln_used(r, s) && ln_e(s) <= EMAX) Z[r][s] = fmaf(f[r][ln_e(s)], tc.WPN[ln_p(s)][k], Z[r][s]);
}

template <int LW>
__global__ void __launch_bounds__(32 * LW, 6) k_predict_lines(Geo q, Region box, const float* __restrict__ W,
                                                           const double* __restrict__ d_dt, int picard,
                                                           float* __restrict__ FS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kTB = ((sizeof(Tabs<float>) + 15) / 16) * 16;
  constexpr int kIX = ((sizeof(LineIdx) + 15) / 16) * 16;
  Tabs<float>& tb = *reinterpret_cast<Tabs<float>*>(smem_raw);
  LineIdx& ix = *reinterpret_cast<LineIdx*>(smem_raw + kTB);
  float* smem = reinterpret_cast<float*>(smem_raw + kTB + kIX);
  {
    const int* src = reinterpret_cast<const int*>(&tabs<float>(3));
    int* dst = reinterpret_cast<int*>(&tb);
    for (int i = threadIdx.x; i < (int)(sizeof(Tabs<float>) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    const int8_t* s8 = reinterpret_cast<const int8_t*>(&c_lidx);
    int8_t* d8 = reinterpret_cast<int8_t*>(&ix);
    for (int i = threadIdx.x; i < (int)sizeof(LineIdx); i += blockDim.x) d8[i] = s8[i];
  }
  __syncthreads();
  const Tabs<float>& tc = tabs<float>(3);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int zh = lane >> 4, l16 = lane & 15;
  const int li = l16 & 3, lj = l16 >> 2;   // this lane's line of nodes (x_i, y_j, z_0..3)
  float* wbase = smem + wib * LineSmem::SIZE;
  float* sw = wbase + LineSmem::W + zh * LineSmem::WS;
  float* sg = wbase + LineSmem::G + zh * LineSmem::GS;
  float* y2 = wbase + LineSmem::Y2 + zh * LineSmem::Y2S;
  float* y3 = wbase + LineSmem::Y3 + zh * LineSmem::Y3S;
  const long long nb = box.size();
  const double dt = *d_dt;
  float lam[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) lam[d] = (float)(dt / q.dx[d]);
  const float gm1 = (float)(q.gamma - 1.0);
  // P_a(x_i) P_b(y_j) at this lane's line, a + b <= 3
  float phi[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4 - a; ++b) phi[a][b] = tb.PN[a][li] * tb.PN[b][lj];

  // the modes of the next zone pair are loaded while this one is computed
  // (a zone beyond the box reads a uniform state and stores nothing)
  constexpr int ZPB = 2 * LW;   // zones per block, consecutive
  const long long rstep = (long long)gridDim.x * ZPB;
  __shared__ unsigned char s_bad[ZPB];   // positivity fallback per zone of the block
  float wpre[7];
  auto fetch = [&](long long rr) {
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const int it = l16 + 16 * k;
      wpre[k] = it < 100 && rr < nb ? W[(long long)it * nb + rr] : (it == 0 || it == 80 ? 1.f : 0.f);
    }
  };
  // the loop is uniform over the block (its zones are stored together at the
  // end of an iteration); zones beyond the box compute on the uniform state
  long long r0 = (long long)blockIdx.x * ZPB + 2 * wib;
  fetch(r0 + zh);
  for (long long rb = (long long)blockIdx.x * ZPB; rb < nb; rb += rstep, r0 += rstep) {
    const bool live = r0 + zh < nb;   // this lane's zone exists
#pragma unroll
    for (int k = 0; k < 7; ++k)
      if (l16 + 16 * k < 100) sw[l16 + 16 * k] = wpre[k];
    fetch(r0 + rstep + zh);
    for (int it = l16; it < 80; it += 16) sg[it] = 0.f;
    __syncwarp();
    // w at the line's four nodes: contract x and y (a + b <= 3 - c), then z
    float wn[5][4];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float wv[20];
#pragma unroll
      for (int k4 = 0; k4 < 5; ++k4) {
        const float4 t4 = *reinterpret_cast<const float4*>(sw + v * 20 + 4 * k4);
        wv[4 * k4] = t4.x; wv[4 * k4 + 1] = t4.y; wv[4 * k4 + 2] = t4.z; wv[4 * k4 + 3] = t4.w;
      }
      float w2[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b <= 3 - c; ++b)
#pragma unroll
          for (int a = 0; a <= 3 - b - c; ++a) acc = fmaf(wv[simplex_idx(3, a, b, c)], phi[a][b], acc);
        w2[c] = acc;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float acc = w2[0] * tc.PN[0][k];
#pragma unroll
        for (int c = 1; c < 4; ++c) acc = fmaf(w2[c], tc.PN[c][k], acc);
        wn[v][k] = acc;
      }
    }
    if (picard >= 1) {
      // sweep 0: time-independent flux at the spatial nodes
      float Z[9][9];
#pragma unroll
      for (int rr = 0; rr < 9; ++rr)
#pragma unroll
        for (int s = 0; s < 9; ++s) Z[rr][s] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float qn[5], f1[9], f[9][3];
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = wn[v][k];
        sym_fluxes<float>(qn, __fdividef(1.f, qn[0]), gm1, f1);   // as recip_pair
#pragma unroll
        for (int rr = 0; rr < 9; ++rr) f[rr][0] = f[rr][1] = f[rr][2] = f1[rr];
        line_z_accumulate<0>(Z, f, k);
      }
#pragma unroll
      for (int rr = 0; rr < 9; ++rr)
#pragma unroll
        for (int s = 0; s < 9; ++s)
          if (ln_used(rr, s) && ln_e(s) == 0) y2[ln_rowbase(rr) + s * 16 + l16] = Z[rr][s];
      __syncwarp();
      line_project<0>(y2, y3, sg, sw, tb, ix, l16, lam);
    }
    for (int sweep = 1; sweep < picard; ++sweep) {
      // The iterate's correction along the line: with H_ce = sum_{a,b} g_abce
      // P_a(x_i) P_b(y_j), the z-mode 0 part at the four time nodes,
      // C0[v][t] = sum_e H_0e I_e(tau_t), and the z-mode 1, 2 coefficients H_10,
      // H_11, H_20, whose products with I_e(tau_t) P_c(z_k) are constants
      float C0[5][4], H1[5][3];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        float gv[16];
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
          const float4 t4 = *reinterpret_cast<const float4*>(sg + v * 16 + 4 * k4);
          gv[4 * k4] = t4.x; gv[4 * k4 + 1] = t4.y; gv[4 * k4 + 2] = t4.z; gv[4 * k4 + 3] = t4.w;
        }
        float H[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int e = 0; e <= 2 - c; ++e) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; b <= 2 - c - e; ++b)
#pragma unroll
              for (int a = 0; a <= 2 - b - c - e; ++a) acc = fmaf(gv[gmidx(a, b, c, e)], phi[a][b], acc);
            H[c][e] = acc;
          }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          float acc = H[0][0] * tc.IT[0][t];
          acc = fmaf(H[0][1], tc.IT[1][t], acc);
          C0[v][t] = fmaf(H[0][2], tc.IT[2][t], acc);
        }
        H1[v][0] = H[1][0];
        H1[v][1] = H[1][1];
        H1[v][2] = H[2][0];
      }
      float Z[9][9];
#pragma unroll
      for (int rr = 0; rr < 9; ++rr)
#pragma unroll
        for (int s = 0; s < 9; ++s) Z[rr][s] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        NodeAcc<float> acc = {};
#pragma unroll
        for (int tp = 0; tp < 2; ++tp) {
          float f[2][9], qn[2][5];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int t = h ? 3 - tp : tp;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              float x = wn[v][k] - C0[v][t];   // P_0 = 1
#pragma unroll
              for (int j = 0; j < 3; ++j) x = fmaf(-H1[v][j], c_ln_itpn[j][t][k], x);
              qn[h][v] = x;
            }
          }
          float ia, ib;
          recip_pair<float>(qn[0][0], qn[1][0], ia, ib);
          sym_fluxes<float>(qn[0], ia, gm1, f[0]);
          sym_fluxes<float>(qn[1], ib, gm1, f[1]);
          accumulate_pair<float>(acc, f[0], f[1], tc, tp);
        }
        line_z_accumulate<2>(Z, acc.a, k);
      }
#pragma unroll
      for (int rr = 0; rr < 9; ++rr)
#pragma unroll
        for (int s = 0; s < 9; ++s)
          if (ln_used(rr, s)) y2[ln_rowbase(rr) + s * 16 + l16] = Z[rr][s];
      __syncwarp();
      line_project<2>(y2, y3, sg, sw, tb, ix, l16, lam);
    }
    // Face values of the warp's two zones at once: lane l16 of a zone takes the
    // (variable, direction-side) combinations l16 and l16 + 16 (< 30); the
    // zone's z-projected flux rows are dead and hold the face values (240) and
    // the time-integrated G (100)
    face_gt_vt<float, 16>(sg, y2 + 240, tb, l16);
    __syncwarp();
    {
      // both combinations evaluated before either is stored, so that their
      // independent chains interleave (lanes 14, 15 repeat combination 29
      // and store only their first)
      const int c0 = l16, c1 = l16 + 16 < 30 ? l16 + 16 : 29;
      float o0[8], o1[8];
      face_values_reg<float>(sw, y2 + 240, tb, c0 % 5, c0 / 5, o0);
      face_values_reg<float>(sw, y2 + 240, tb, c1 % 5, c1 / 5, o1);
      face_values_store<float>(y2, c0 % 5, c0 / 5, o0);
      if (l16 + 16 < 30) face_values_store<float>(y2, c1 % 5, c1 / 5, o1);
    }
    __syncwarp();
    bool bad = false;
    if (q.fallback)
      for (int row = l16; row < 48; row += 16) bad = bad || !state_physical5<float>(y2 + row * 5, gm1);
    const unsigned ballot = __ballot_sync(0xffffffffu, bad);
    const bool zbad = q.fallback && live && ((ballot >> (16 * zh)) & 0xffffu) != 0;
    if (l16 == 0) s_bad[2 * wib + zh] = zbad ? 1 : 0;
    if (zbad && l16 == 0 && q.fb_count) atomicAdd(q.fb_count, 1ULL);
    __syncthreads();
    // the block's consecutive zones stored together: neighbouring threads write
    // neighbouring zones of one (face row, variable), so a warp's store covers
    // eight entries of four zones instead of 32 entries of one
    for (int it = threadIdx.x; it < 240 * ZPB; it += blockDim.x) {
      const int zb = it % ZPB, e = it / ZPB;
      const long long rz = rb + zb;
      if (rz < nb) {
        const float* zw = smem + (zb >> 1) * LineSmem::SIZE;
        const int zz = zb & 1;
        FS[(long long)e * nb + rz] = s_bad[zb] ? zw[LineSmem::W + zz * LineSmem::WS + (e % 5) * 20]
                                               : zw[LineSmem::Y2 + zz * LineSmem::Y2S + e];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
static bool g_fact_tables_ready = false;

static cudaError_t upload_fact_indices(cudaStream_t s) {
  FactIdx h;
  auto g = st_modes(3, 2);
  // mass-row sources (mass_gmode): the momentum mode one degree up in d, and
  // for b = 0 the mode three degrees up (dP3 = 3 P2 + P0/10)
  memset(h.mass_src, 255, sizeof(h.mass_src));
  for (int d = 0; d < 3; ++d)
    for (int b = 0; b < 16; ++b) h.mass_src[d][5][b] = 0;
  for (int b = 0; b < 15; ++b) {
    const int e = g[b][3];
    for (int d = 0; d < 3; ++d) {
      for (int k = 0; k < 2; ++k) {
        int abc[3] = {g[b][0], g[b][1], g[b][2]};
        const int ad = abc[d];
        if (k == 1 && ad != 0) break;
        abc[d] = k == 0 ? ad + 1 : 3;
        const int deg = abc[0] + abc[1] + abc[2];
        if (deg + e > 3) continue;
        if (k == 1) {
          h.mass_src[d][4][b] = (uint8_t)((1 + d) * 20 + simplex_idx(3, abc[0], abc[1], abc[2]));
          continue;
        }
        h.mass_src[d][5][b] = (uint8_t)(ad + 1);
        h.mass_src[d][0][b] = (uint8_t)((1 + d) * 20 + simplex_idx(3, abc[0], abc[1], abc[2]));
        for (int ee = 0; ee < 3; ++ee)
          if (deg + ee <= 2) h.mass_src[d][1 + ee][b] = (uint8_t)((1 + d) * 15 + gmidx(abc[0], abc[1], abc[2], ee));
      }
    }
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_fidx, &h, sizeof(h), 0, cudaMemcpyHostToDevice, s);
  // the same sources for the line kernel, whose g rows are 16 floats apart
  LineIdx hl;
  memset(&hl, 0, sizeof(hl));
  for (int d = 0; d < 3; ++d)
    for (int b = 0; b < 16; ++b) {
      const uint8_t ow = h.mass_src[d][0][b], o3 = h.mass_src[d][4][b];
      hl.ms_off[d][0][b] = ow != 255 ? ow : 0;
      for (int k = 1; k <= 3; ++k) {
        const uint8_t o = h.mass_src[d][k][b];
        hl.ms_off[d][k][b] = o != 255 ? (uint8_t)((o / 15) * 16 + o % 15) : 15;
      }
      hl.ms_off[d][4][b] = o3 != 255 ? o3 : 0;
      hl.ms_fac[d][b] = (float)h.mass_src[d][5][b];   // 0 where ow is missing
      hl.ms_c3[d][b] = o3 != 255 ? 0.1f : 0.f;
    }
  for (int b = 0; b < 15; ++b) {
    const int ee = g[b][3];
    hl.ms_coef[b][0] = ee == 0 ? 1.f : 0.f;
    hl.ms_coef[b][1] = ee == 2 ? 0.f : -0.5f;
    hl.ms_coef[b][2] = ee == 0 ? 1.f / 6.f : ee == 2 ? -1.f / 6.f : 0.f;
    hl.ms_coef[b][3] = ee == 1 ? 0.1f : 0.f;
    hl.lp_cfac[b] = (float)(g[b][2] + 1);
  }
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_lidx, &hl, sizeof(hl), 0, cudaMemcpyHostToDevice, s);
  {
    Tabs<double> td[3];
    Tabs<float> tf[3];
    build_tabs(td, tf);
    float itpn[3][4][4];
    const int ce[3][2] = {{1, 0}, {1, 1}, {2, 0}};
    for (int j = 0; j < 3; ++j)
      for (int t = 0; t < 4; ++t)
        for (int k = 0; k < 4; ++k) itpn[j][t][k] = (float)(td[2].IT[ce[j][1]][t] * td[2].PN[ce[j][0]][k]);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_ln_itpn, itpn, sizeof(itpn), 0, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

template <typename T> static size_t fact_smem(int wpb) {
  return ((sizeof(Tabs<T>) + 15) / 16) * 16 + ((sizeof(FactIdx) + 15) / 16) * 16 +
         (size_t)wpb * FactSmem<T>::SIZE * sizeof(T);
}
constexpr int kFactWarpsD = 2;   // FP64: two zones per block, four blocks per SM
constexpr int kFactWarpsF = 2;   // FP32 (factorised kernel; the line kernel replaces it)
constexpr int kLineWarps = 2;    // FP32 line kernel: four zones per block
static size_t line_smem(int lw) {
  return ((sizeof(Tabs<float>) + 15) / 16) * 16 + ((sizeof(LineIdx) + 15) / 16) * 16 +
         (size_t)lw * LineSmem::SIZE * sizeof(float);
}

cudaError_t predict_init(cudaStream_t s) {
  if (g_fact_tables_ready) return cudaSuccess;
  cudaError_t e = upload_local_tables(s);
  if (e == cudaSuccess) e = upload_fact_indices(s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_predict_fact<double, kFactWarpsD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fact_smem<double>(kFactWarpsD));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_predict_fact<float, kFactWarpsF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fact_smem<float>(kFactWarpsF));
  // as much shared memory as the SM has: the block count per SM is set by it
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_predict_fact<double, kFactWarpsD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_predict_fact<float, kFactWarpsF>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_predict_lines<kLineWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)line_smem(kLineWarps));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_predict_lines<kLineWarps>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) g_fact_tables_ready = true;
  return e;
}

void launch_predict_tab(const Geo& q, int prec, int picard, const void* W, const double* d_dt,
                        int z0, int z1, const void* tab, const PTabLayout& L, void* FS,
                        cudaStream_t s) {
  Region box = region_box(q, z0, z1);
  long long nb = box.size();
  if (q.dim == 3 && q.N == 3) {
    if (prec == AWE_FP64) {
      long long blocks = (nb + kFactWarpsD - 1) / kFactWarpsD;
      if (blocks > 152LL * 256) blocks = 152LL * 256;
      k_predict_fact<double, kFactWarpsD><<<(int)blocks, 32 * kFactWarpsD, fact_smem<double>(kFactWarpsD), s>>>(
          q, box, (const double*)W, d_dt, picard, (const double*)tab, L, (double*)FS);
    } else {
      const long long zpb = 2 * kLineWarps;   // zones per block
      long long blocks = (nb + zpb - 1) / zpb;
      if (blocks > 152LL * 256) blocks = 152LL * 256;
      k_predict_lines<kLineWarps><<<(int)blocks, 32 * kLineWarps, line_smem(kLineWarps), s>>>(
          q, box, (const float*)W, d_dt, picard, (float*)FS);
    }
    return;
  }
  const int th = 128;
  long long blocks = (nb + th - 1) / th;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
#define AWE_PD(D_, N_)                                                                           \
  if (q.dim == D_ && q.N == N_) {                                                                \
    if (prec == AWE_FP64)                                                                        \
      k_predict_direct<D_, N_, double><<<(int)blocks, th, 0, s>>>(q, box, (const double*)W, d_dt,  \
                                                                  picard, (const double*)tab, L, \
                                                                  (double*)FS);                  \
    else                                                                                         \
      k_predict_direct<D_, N_, float><<<(int)blocks, th, 0, s>>>(q, box, (const float*)W, d_dt,    \
                                                                 picard, (const float*)tab, L,   \
                                                                 (float*)FS);                    \
    return;                                                                                      \
  }
  AWE_PD(2, 1)
  AWE_PD(2, 2)
  AWE_PD(2, 3)
  AWE_PD(3, 1)
  AWE_PD(3, 2)
#undef AWE_PD
}

}  // namespace awe
