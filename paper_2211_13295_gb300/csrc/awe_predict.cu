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

namespace awe {

// ---------------------------------------------------------------------------
// direct predictor
// ---------------------------------------------------------------------------
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
      // sweep 0: time-independent flux at the spatial nodes
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
          for (int v = 0; v < NV; ++v) {
            T f = lam[d] * F[d][v];
#pragma unroll
            for (int b = 0; b < NG0; ++b) g[v][b] = fma(f, ks[b], g[v][b]);
          }
        }
      }
      for (int sweep = 1; sweep < picard; ++sweep) {
        T gn[NV][NG];
#pragma unroll
        for (int v = 0; v < NV; ++v)
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
          for (int t = 0; t < NN; ++t) {
            const int node = s * NN + t;
            const T* ev = EV + (long long)node * NG;
            T qn[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              T acc = wn[v];
#pragma unroll
              for (int b = 0; b < NG; ++b) acc = fma(-g[v][b], ev[b], acc);
              qn[v] = acc;
            }
            T F[D][D + 2];
            phys_fluxes<D, T>(qn, gm1, F);
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const T* kp = KP + ((long long)d * (NSN * NN) + node) * NG;
#pragma unroll
              for (int v = 0; v < NV; ++v) {
                T f = lam[d] * F[d][v];
#pragma unroll
                for (int b = 0; b < NG; ++b) gn[v][b] = fma(f, kp[b], gn[v][b]);
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
    // face quadrature states: q = w(face point) - int_0^tau G
    for (int row = 0; row < D * 2 * NFQ; ++row) {
      const T* fw = FW + (long long)row * NS;
      const T* fg = FG + (long long)row * NG;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < NS; ++m) acc = fma(w[v][m], fw[m], acc);
#pragma unroll
        for (int b = 0; b < NG; ++b) acc = fma(-g[v][b], fg[b], acc);
        FS[((long long)row * NV + v) * nb + r] = acc;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// factorised predictor, 3D, N = 3: one warp per zone
// ---------------------------------------------------------------------------
// index tables (constant memory): see the stage comments
__constant__ int8_t c_sm3[20][3];     // spatial modes degree <= 3, (a,b,c)
__constant__ int8_t c_pair3[10][2];   // (b,c) with b+c <= 3, c outer
__constant__ int8_t c_tri2[10][3];    // (p,q,r) with p+q+r <= 2, r outer, q, p inner
__constant__ int8_t c_pair2[6][2];    // (p,e) with p+e <= 2, e outer
__constant__ int8_t c_gm[15][4];      // G-modes (a,b,c,e), degree <= 2, e outermost
__constant__ int8_t c_gidx[3][3][3][3];  // (a,b,c,e) -> G-mode index, -1 outside
__constant__ int8_t c_tri_idx[3][3][3];  // (p,q,r) -> index in c_tri2
__constant__ int8_t c_pair2_idx[3][3];   // (p,e) -> index in c_pair2
__constant__ int8_t c_pair3_idx[4][4];   // (b,c) -> index in c_pair3
__constant__ int8_t c_sm3_idx[4][4][4];  // (a,b,c) -> spatial mode index

template <typename T> struct FactSmem {
  // per-zone layout (elements of T)
  static constexpr int W = 0;                  // w[5][20]
  static constexpr int WN = W + 100;           // wn[5][64]
  static constexpr int G = WN + 320;           // g[5][15]
  static constexpr int R1 = G + 75;            // T1/T2, A/B/C, Y2 (max 1640)
  static constexpr int R2 = R1 + 1640;         // Y1 (2880), Y3 (600)
  static constexpr int SIZE = R2 + 2880;       // 5015
};

template <typename T, int EMAX>
__device__ __forceinline__ void fact_project(T* z, const Tabs<T>& tb, int lane, const T lam[3]) {
  constexpr int NPE = EMAX == 0 ? 3 : 6;     // (p,e) pairs with e <= EMAX
  constexpr int NTR = EMAX == 0 ? 6 : 10;    // (p,q,e) triples with e <= EMAX
  constexpr int NGE = EMAX == 0 ? 10 : 15;   // G-modes with e <= EMAX
  T* Y1 = z + FactSmem<T>::R2;               // [d][v][s][e3]  (e3 stride 3)
  T* Y2 = z + FactSmem<T>::R1;               // [d][v][n2][pe] (pe stride 6)
  T* Y3 = z + FactSmem<T>::R2;               // [d][v][n1][tri] (tri stride 10)
  // P1: contract the first dimension (z for d = x, y; y for d = z)
  for (int it = lane; it < 3 * 5 * 16 * NPE; it += 32) {
    int pe = it % NPE;
    int rest = it / NPE;
    int n2 = rest % 16;
    int dv = rest / 16;  // d*5 + v
    int d = dv / 5;
    int p = c_pair2[pe][0], e = c_pair2[pe][1];
    int a0 = n2 & 3, a1 = n2 >> 2;
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      // d < 2: n2 = (i,j), sum over k; d = 2: n2 = (i,k), sum over j
      int s = d < 2 ? (a0 + 4 * a1 + 16 * m) : (a0 + 4 * m + 16 * a1);
      acc = fma(Y1[(dv * 64 + s) * 3 + e], tb.WPN[p][m], acc);
    }
    Y2[(dv * 16 + n2) * 6 + pe] = acc;
  }
  __syncwarp();
  // P2: contract the second dimension (y for d = x; x for d = y, z)
  for (int it = lane; it < 3 * 5 * 4 * NTR; it += 32) {
    int tr = it % NTR;
    int rest = it / NTR;
    int n1 = rest % 4;
    int dv = rest / 4;
    int d = dv / 5;
    int p = c_tri2[tr][0], qq = c_tri2[tr][1], e = c_tri2[tr][2];
    // d = x: Y3[i][(b,c,e)] = sum_j Y2[(i,j)][(c,e)] WPN[b][j]      (p=b, qq=c)
    // d = y: Y3[j][(a,c,e)] = sum_i Y2[(i,j)][(c,e)] WPN[a][i]      (p=a, qq=c)
    // d = z: Y3[k][(a,b,e)] = sum_i Y2[(i,k)][(b,e)] WPN[a][i]      (p=a, qq=b)
    int pe = c_pair2_idx[qq][e];
    T acc = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      int n2 = d == 0 ? (n1 + 4 * m) : (m + 4 * n1);
      acc = fma(Y2[(dv * 16 + n2) * 6 + pe], tb.WPN[p][m], acc);
    }
    Y3[(dv * 4 + n1) * 10 + tr] = acc;
  }
  __syncwarp();
  // P3: contract the derivative dimension with the Q factors, sum over d
  for (int it = lane; it < 5 * NGE; it += 32) {
    int b = it % NGE;
    int v = it / NGE;
    int a = c_gm[b][0], bb = c_gm[b][1], c = c_gm[b][2], e = c_gm[b][3];
    int slack = 3 - (a + bb + c + e);
    T acc = T(0);
    int t0 = c_tri_idx[bb][c][e], t1 = c_tri_idx[a][c][e], t2 = c_tri_idx[a][bb][e];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      acc = fma(lam[0] * Y3[((0 * 5 + v) * 4 + m) * 10 + t0], tb.QN[a][slack][m], acc);
      acc = fma(lam[1] * Y3[((1 * 5 + v) * 4 + m) * 10 + t1], tb.QN[bb][slack][m], acc);
      acc = fma(lam[2] * Y3[((2 * 5 + v) * 4 + m) * 10 + t2], tb.QN[c][slack][m], acc);
    }
    z[FactSmem<T>::G + v * 15 + b] = acc;
  }
  if (EMAX == 0) {
    for (int it = lane; it < 5 * 5; it += 32) z[FactSmem<T>::G + (it / 5) * 15 + 10 + it % 5] = T(0);
  }
  __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(128) k_predict_fact(Geo q, Region box, const T* __restrict__ W,
                                                      const double* __restrict__ d_dt, int picard,
                                                      const T* __restrict__ tab, PTabLayout L,
                                                      T* __restrict__ FS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  T* z = smem + wib * FactSmem<T>::SIZE;
  const Tabs<T>& tb = tabs<T>(3);
  const long long nb = box.size();
  const double dt = *d_dt;
  T lam[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) lam[d] = (T)(dt / q.dx[d]);
  const T gm1 = (T)(q.gamma - 1.0);
  const T* FW = tab + L.fw;
  const T* FG = tab + L.fg;
  for (long long r = (long long)blockIdx.x * wpb + wib; r < nb; r += (long long)gridDim.x * wpb) {
    T* sw = z + FactSmem<T>::W;
    T* swn = z + FactSmem<T>::WN;
    T* sg = z + FactSmem<T>::G;
    for (int it = lane; it < 100; it += 32) sw[it] = W[(long long)it * nb + r];
    __syncwarp();
    // w at the 64 spatial nodes: contract a, then b, then c
    {
      T* T1 = z + FactSmem<T>::R1;        // [v][i][pair3]   200
      T* T2 = T1 + 200;                   // [v][i][j][c]    320
      for (int it = lane; it < 200; it += 32) {
        int pc = it % 10, rest = it / 10, i = rest % 4, v = rest / 4;
        int b = c_pair3[pc][0], c = c_pair3[pc][1];
        T acc = T(0);
        for (int a = 0; a <= 3 - b - c; ++a) acc = fma(sw[v * 20 + c_sm3_idx[a][b][c]], tb.PN[a][i], acc);
        T1[it] = acc;
      }
      __syncwarp();
      for (int it = lane; it < 320; it += 32) {
        int c = it % 4, rest = it / 4, j = rest % 4, rest2 = rest / 4, i = rest2 % 4, v = rest2 / 4;
        T acc = T(0);
        for (int b = 0; b <= 3 - c; ++b) acc = fma(T1[(v * 4 + i) * 10 + c_pair3_idx[b][c]], tb.PN[b][j], acc);
        T2[it] = acc;
      }
      __syncwarp();
      for (int it = lane; it < 320; it += 32) {
        int s = it % 64, v = it / 64;
        int i = s & 3, j = (s >> 2) & 3, k = s >> 4;
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc = fma(T2[((v * 4 + i) * 4 + j) * 4 + c], tb.PN[c][k], acc);
        swn[v * 64 + s] = acc;
      }
      __syncwarp();
    }
    for (int it = lane; it < 75; it += 32) sg[it] = T(0);
    __syncwarp();
    T* Y1 = z + FactSmem<T>::R2;
    if (picard >= 1) {
      // sweep 0: flux at the spatial nodes, time-independent
      for (int s = lane; s < 64; s += 32) {
        T qn[5], F[3][5];
#pragma unroll
        for (int v = 0; v < 5; ++v) qn[v] = swn[v * 64 + s];
        phys_fluxes<3, T>(qn, gm1, F);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v) Y1[((d * 5 + v) * 64 + s) * 3 + 0] = F[d][v];
      }
      __syncwarp();
      fact_project<T, 0>(z, tb, lane, lam);
    }
    for (int sweep = 1; sweep < picard; ++sweep) {
      T* A = z + FactSmem<T>::R1;   // [v][tri][t]        200
      T* B = A + 200;               // [v][i][pair2][t]   480
      T* C = B + 480;               // [v][i][j][c][t]    960
      // E1: A[v][(a,b,c)][t] = sum_e g[(a,b,c,e)] I_e(tau_t)
      for (int it = lane; it < 200; it += 32) {
        int t = it % 4, rest = it / 4, tr = rest % 10, v = rest / 10;
        int a = c_tri2[tr][0], b = c_tri2[tr][1], c = c_tri2[tr][2];
        T acc = T(0);
        for (int e = 0; e <= 2 - a - b - c; ++e) acc = fma(sg[v * 15 + c_gidx[a][b][c][e]], tb.IT[e][t], acc);
        A[it] = acc;
      }
      __syncwarp();
      // E2: B[v][i][(b,c)][t] = sum_a A[(a,b,c)][t] P_a(x_i)
      for (int it = lane; it < 480; it += 32) {
        int t = it % 4, rest = it / 4, pc = rest % 6, rest2 = rest / 6, i = rest2 % 4, v = rest2 / 4;
        int b = c_pair2[pc][0], c = c_pair2[pc][1];
        T acc = T(0);
        for (int a = 0; a <= 2 - b - c; ++a) acc = fma(A[(v * 10 + c_tri_idx[a][b][c]) * 4 + t], tb.PN[a][i], acc);
        B[it] = acc;
      }
      __syncwarp();
      // E3: C[v][i][j][c][t] = sum_b B[i][(b,c)][t] P_b(y_j)
      for (int it = lane; it < 960; it += 32) {
        int t = it % 4, rest = it / 4, c = rest % 3, rest2 = rest / 3, j = rest2 % 4, rest3 = rest2 / 4;
        int i = rest3 % 4, v = rest3 / 4;
        T acc = T(0);
        for (int b = 0; b <= 2 - c; ++b) acc = fma(B[((v * 4 + i) * 6 + c_pair2_idx[b][c]) * 4 + t], tb.PN[b][j], acc);
        C[it] = acc;
      }
      __syncwarp();
      // nodes: q = wn - sum_c C P_c(z_k); fluxes; time contraction into Y1
      for (int s = lane; s < 64; s += 32) {
        int i = s & 3, j = (s >> 2) & 3, k = s >> 4;
        T acc[3][5][3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int e = 0; e < 3; ++e) acc[d][v][e] = T(0);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          T qn[5], F[3][5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            T x = swn[v * 64 + s];
#pragma unroll
            for (int c = 0; c < 3; ++c) x = fma(-C[((((v * 4 + i) * 4 + j) * 3 + c) * 4) + t], tb.PN[c][k], x);
            qn[v] = x;
          }
          phys_fluxes<3, T>(qn, gm1, F);
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int v = 0; v < 5; ++v)
#pragma unroll
              for (int e = 0; e < 3; ++e) acc[d][v][e] = fma(tb.WLT[e][t], F[d][v], acc[d][v][e]);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int v = 0; v < 5; ++v)
#pragma unroll
            for (int e = 0; e < 3; ++e) Y1[((d * 5 + v) * 64 + s) * 3 + e] = acc[d][v][e];
      }
      __syncwarp();
      fact_project<T, 2>(z, tb, lane, lam);
    }
    // face states
    for (int it = lane; it < 240; it += 32) {
      int v = it % 5, row = it / 5;
      const T* fw = FW + row * 20;
      const T* fg = FG + row * 15;
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < 20; ++m) acc = fma(sw[v * 20 + m], fw[m], acc);
#pragma unroll
      for (int b = 0; b < 15; ++b) acc = fma(-sg[v * 15 + b], fg[b], acc);
      FS[((long long)row * 5 + v) * nb + r] = acc;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
static bool g_fact_tables_ready = false;

static cudaError_t upload_fact_indices(cudaStream_t s) {
  int8_t sm3[20][3], pair3[10][2], tri2[10][3], pair2[6][2], gm[15][4];
  int8_t gidx4[3][3][3][3], tri_idx[3][3][3], pair2_idx[3][3], pair3_idx[4][4], sm3_idx[4][4][4];
  memset(gidx4, -1, sizeof(gidx4));
  memset(tri_idx, -1, sizeof(tri_idx));
  memset(pair2_idx, -1, sizeof(pair2_idx));
  memset(pair3_idx, -1, sizeof(pair3_idx));
  memset(sm3_idx, -1, sizeof(sm3_idx));
  int m = 0;
  for (int c = 0; c <= 3; ++c)
    for (int b = 0; b <= 3 - c; ++b)
      for (int a = 0; a <= 3 - b - c; ++a) {
        sm3[m][0] = a; sm3[m][1] = b; sm3[m][2] = c;
        sm3_idx[a][b][c] = m++;
      }
  m = 0;
  for (int c = 0; c <= 3; ++c)
    for (int b = 0; b <= 3 - c; ++b) {
      pair3[m][0] = b; pair3[m][1] = c;
      pair3_idx[b][c] = m++;
    }
  m = 0;
  for (int r = 0; r <= 2; ++r)
    for (int qq = 0; qq <= 2 - r; ++qq)
      for (int p = 0; p <= 2 - r - qq; ++p) {
        tri2[m][0] = p; tri2[m][1] = qq; tri2[m][2] = r;
        tri_idx[p][qq][r] = m++;
      }
  m = 0;
  for (int e = 0; e <= 2; ++e)
    for (int p = 0; p <= 2 - e; ++p) {
      pair2[m][0] = p; pair2[m][1] = e;
      pair2_idx[p][e] = m++;
    }
  auto g = st_modes(3, 2);
  for (int b = 0; b < 15; ++b) {
    for (int t = 0; t < 4; ++t) gm[b][t] = (int8_t)g[b][t];
    gidx4[g[b][0]][g[b][1]][g[b][2]][g[b][3]] = b;
  }
  cudaError_t e = cudaSuccess;
#define UP(sym, src) if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(sym, src, sizeof(src), 0, cudaMemcpyHostToDevice, s)
  UP(c_sm3, sm3); UP(c_pair3, pair3); UP(c_tri2, tri2); UP(c_pair2, pair2); UP(c_gm, gm);
  UP(c_gidx, gidx4); UP(c_tri_idx, tri_idx); UP(c_pair2_idx, pair2_idx); UP(c_pair3_idx, pair3_idx);
  UP(c_sm3_idx, sm3_idx);
#undef UP
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t predict_init(cudaStream_t s) {
  if (g_fact_tables_ready) return cudaSuccess;
  cudaError_t e = upload_local_tables(s);
  if (e == cudaSuccess) e = upload_fact_indices(s);
  if (e == cudaSuccess) {
    size_t smd = 4 * FactSmem<double>::SIZE * sizeof(double);
    size_t smf = 4 * FactSmem<float>::SIZE * sizeof(float);
    e = cudaFuncSetAttribute(k_predict_fact<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_predict_fact<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
  }
  if (e == cudaSuccess) g_fact_tables_ready = true;
  return e;
}

void launch_predict_tab(const Geo& q, int prec, int picard, const void* W, const double* d_dt,
                        int z0, int z1, const void* tab, const PTabLayout& L, void* FS,
                        cudaStream_t s) {
  Region box = region_box(q, z0, z1);
  long long nb = box.size();
  if (q.dim == 3 && q.N == 3) {
    const int wpb = 4;
    long long blocks = (nb + wpb - 1) / wpb;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    if (prec == AWE_FP64)
      k_predict_fact<double><<<(int)blocks, 32 * wpb, wpb * FactSmem<double>::SIZE * sizeof(double), s>>>(
          q, box, (const double*)W, d_dt, picard, (const double*)tab, L, (double*)FS);
    else
      k_predict_fact<float><<<(int)blocks, 32 * wpb, wpb * FactSmem<float>::SIZE * sizeof(float), s>>>(
          q, box, (const float*)W, d_dt, picard, (const float*)tab, L, (float*)FS);
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
  AWE_PD(2, 2)
  AWE_PD(2, 3)
  AWE_PD(3, 2)
#undef AWE_PD
}

}  // namespace awe
