// awe_rk.cu -- the Runge-Kutta variant of the step, the time stepping the
// paper compares ADER with (Table IV: two stages at second order, three at
// third, five at fourth).  Per stage: the reconstruction of the stage state
// (awe_recon.cu), its values at the face Gauss points (no predictor), the
// face-averaged Riemann fluxes (awe_flux.cuh with the face points only) and
// the FP64 stage combination of the Shu-Osher form
//   U(i) = sum_{k<i} [ alpha_ik U(k) + beta_ik dt L(U(k)) ],
//   L(U) = -sum_d (F_{d,i+1/2} - F_{d,i-1/2}) / dx_d,
// for SSP(2,2) (Heun), SSP(3,3) (Shu and Osher) and the five-stage,
// fourth-order SSP(5,4) of Spiteri and Ruuth.
#include "awe_flux.cuh"
#include "awe_rk.h"

namespace awe {

bool rk_scheme(int stages, RKScheme& r) {
  for (int i = 0; i <= kRKMax; ++i) {
    r.c[i] = 0.0;
    for (int k = 0; k < kRKMax; ++k) r.alpha[i][k] = r.beta[i][k] = 0.0;
  }
  r.s = stages;
  if (stages == 2) {
    r.alpha[1][0] = 1.0, r.beta[1][0] = 1.0;
    r.alpha[2][0] = 0.5, r.alpha[2][1] = 0.5, r.beta[2][1] = 0.5;
  } else if (stages == 3) {
    r.alpha[1][0] = 1.0, r.beta[1][0] = 1.0;
    r.alpha[2][0] = 0.75, r.alpha[2][1] = 0.25, r.beta[2][1] = 0.25;
    r.alpha[3][0] = 1.0 / 3.0, r.alpha[3][2] = 2.0 / 3.0, r.beta[3][2] = 2.0 / 3.0;
  } else if (stages == 5) {
    // Spiteri and Ruuth's SSP(5,4), SSP coefficient 1.508
    r.alpha[1][0] = 1.0;
    r.beta[1][0] = 0.391752226571890;
    r.alpha[2][0] = 0.444370493651235, r.alpha[2][1] = 0.555629506348765;
    r.beta[2][1] = 0.368410593050371;
    r.alpha[3][0] = 0.620101851488403, r.alpha[3][2] = 0.379898148511597;
    r.beta[3][2] = 0.251891774271694;
    r.alpha[4][0] = 0.178079954393132, r.alpha[4][3] = 0.821920045606868;
    r.beta[4][3] = 0.544974750228521;
    r.alpha[5][2] = 0.517231671970585, r.alpha[5][3] = 0.096059710526147;
    r.beta[5][3] = 0.063692468666290;
    r.alpha[5][4] = 0.386708617503269, r.beta[5][4] = 0.226007483236906;
  } else {
    return false;
  }
  // stage abscissae: U(i) approximates U(t + c_i dt)
  for (int i = 1; i <= stages; ++i)
    for (int k = 0; k < i; ++k) r.c[i] += r.alpha[i][k] * r.c[k] + r.beta[i][k];
  return true;
}

// ---------------------------------------------------------------------------
// face states of the reconstructed polynomial (no time evolution)
// ---------------------------------------------------------------------------
// FS[d][side][p][var][box zone], p = i1 + nq*i2 < NP (face points only, the
// ADER face point order at the first time point).  Factorised per direction
// d: the normal axis at +-1/2 first, split into the even and odd Legendre
// terms (P_a(-1/2) = (-1)^a P_a(1/2)), which gives both sides at once; then
// the transverse axes at their Gauss nodes +-g, again by parity.  With the
// positivity fallback a zone with a non-physical face state uses its zone mean
// at every face point.
template <typename T> struct FaceConsts {
  T ph[4];  // P_a(1/2)
  T pg[4];  // P_p at the upper transverse Gauss node (0 with one node)
};

// index of the spatial mode with exponents (e0, e1, e2) (c outermost, a innermost)
template <int D, int N>
__host__ __device__ constexpr int face_mode_index(int e0, int e1, int e2) {
  int idx = 0;
  if (D == 3)
    for (int c = 0; c < e2; ++c) idx += (N - c + 1) * (N - c + 2) / 2;
  const int M = D == 3 ? N - e2 : N;
  for (int b = 0; b < e1; ++b) idx += M - b + 1;
  return idx + e0;
}
// mode of normal exponent an and transverse exponents (p1, p2) for direction d
// (t1 < t2 the transverse dimensions)
template <int D, int N>
__host__ __device__ constexpr int face_mode(int d, int an, int p1, int p2) {
  return D == 2 ? (d == 0 ? face_mode_index<D, N>(an, p1, 0) : face_mode_index<D, N>(p1, an, 0))
                : (d == 0 ? face_mode_index<D, N>(an, p1, p2)
                          : d == 1 ? face_mode_index<D, N>(p1, an, p2) : face_mode_index<D, N>(p1, p2, an));
}
// transverse exponent pairs (p1, p2), p1 + p2 <= N, p2 outermost (3D), or p1 (2D)
template <int N> __host__ __device__ constexpr int pair_index(int p1, int p2) {
  return p2 * (N + 1) - p2 * (p2 - 1) / 2 + p1;
}

template <int D, int N, typename T>
__global__ void __launch_bounds__(128) k_face_eval(Geo q, Region box, const T* __restrict__ W,
                                                   FaceConsts<T> fc, T* __restrict__ FS) {
  constexpr int NV = D + 2, NS = Modes<D, N>::NS, NQ = Modes<D, N>::NQ;
  constexpr int NP = kPoints<D, N, true>();
  constexpr int NPAIR = D == 3 ? (N + 1) * (N + 2) / 2 : N + 1;
  constexpr int P2MAX = D == 3 ? N : 0;
  const long long nb = box.size();
  const T gm1 = (T)(q.gamma - 1.0);
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nb;
       r += (long long)gridDim.x * blockDim.x) {
#pragma unroll 1
    for (int v = 0; v < NV; ++v) {
      T w[NS];
#pragma unroll
      for (int m = 0; m < NS; ++m) w[m] = W[((long long)v * NS + m) * nb + r];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        // normal axis: even and odd parts for every transverse pair
        T E[NPAIR], O[NPAIR];
#pragma unroll
        for (int p2 = 0; p2 <= P2MAX; ++p2)
#pragma unroll
          for (int p1 = 0; p1 <= N - p2; ++p1) {
            T e = T(0), o = T(0);
#pragma unroll
            for (int an = 0; an <= N - p1 - p2; ++an) {
              const T x = w[face_mode<D, N>(d, an, p1, p2)];
              if (an & 1) o = fma(x, fc.ph[an], o);
              else e = an == 0 ? x : fma(x, fc.ph[an], e);
            }
            E[pair_index<N>(p1, p2)] = e;
            O[pair_index<N>(p1, p2)] = o;
          }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          // transverse axis t1: V[i1][p2]
          T V[NQ][P2MAX + 1];
#pragma unroll
          for (int p2 = 0; p2 <= P2MAX; ++p2) {
            T ev = T(0), od = T(0);
#pragma unroll
            for (int p1 = 0; p1 <= N - p2; ++p1) {
              const int k = pair_index<N>(p1, p2);
              const T wt = side ? E[k] + O[k] : E[k] - O[k];
              if (p1 & 1) od = fma(wt, fc.pg[p1], od);
              else ev = p1 == 0 ? wt : fma(wt, fc.pg[p1], ev);
            }
            if (NQ == 2) {
              V[0][p2] = ev - od;
              V[NQ - 1][p2] = ev + od;
            } else {
              V[0][p2] = ev;  // at the centre the odd terms vanish
            }
          }
          const long long row0 = (long long)(d * 2 + side) * NP;
          if (D == 2) {
#pragma unroll
            for (int i1 = 0; i1 < NQ; ++i1)
              FS[((row0 + i1) * NV + v) * nb + r] = V[i1][0];
          } else {
            // transverse axis t2
#pragma unroll
            for (int i1 = 0; i1 < NQ; ++i1) {
              T ev = T(0), od = T(0);
#pragma unroll
              for (int p2 = 0; p2 <= P2MAX; ++p2) {
                if (p2 & 1) od = fma(V[i1][p2], fc.pg[p2], od);
                else ev = p2 == 0 ? V[i1][p2] : fma(V[i1][p2], fc.pg[p2], ev);
              }
              if (NQ == 2) {
                FS[((row0 + i1 + NQ * 0) * NV + v) * nb + r] = ev - od;
                FS[((row0 + i1 + NQ * 1) * NV + v) * nb + r] = ev + od;
              } else {
                FS[((row0 + i1) * NV + v) * nb + r] = ev;
              }
            }
          }
        }
      }
    }
    if (q.fallback) {
      constexpr int NR = D * 2 * NP;
      bool bad = false;
      for (int row = 0; row < NR; ++row) {
        T u[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = FS[((long long)row * NV + v) * nb + r];
        bad = bad || !state_physical<D, T>(u, gm1);
      }
      if (bad) {
        if (q.fb_count) atomicAdd(q.fb_count, 1ULL);
#pragma unroll 1
        for (int v = 0; v < NV; ++v) {
          const T mean = W[((long long)v * NS) * nb + r];
          for (int row = 0; row < NR; ++row) FS[((long long)row * NV + v) * nb + r] = mean;
        }
      }
    }
  }
}

template <typename T> static FaceConsts<T> face_consts(int N) {
  FaceConsts<T> c;
  const int nq = (N + 2) / 2;
  double x[4], w[4];
  gauss_nodes(nq, x, w);
  for (int a = 0; a < 4; ++a) {
    c.ph[a] = (T)basisP(a, 0.5);
    c.pg[a] = (T)basisP(a, x[nq - 1]);
  }
  return c;
}

void launch_face_eval(const Geo& q, int prec, const void* W, int z0, int z1, const void* tab,
                      const PTabLayout& L, void* FS, cudaStream_t s) {
  (void)tab;
  (void)L;
  Region box = region_box(q, z0, z1);
  int blocks = grid_for(box.size(), 128, 152LL * 16);
#define AWE_FACE(D_, N_)                                                                   \
  if (q.dim == D_ && q.N == N_) {                                                          \
    if (prec == AWE_FP64)                                                                  \
      k_face_eval<D_, N_, double><<<blocks, 128, 0, s>>>(                                  \
          q, box, (const double*)W, face_consts<double>(N_), (double*)FS);                 \
    else                                                                                   \
      k_face_eval<D_, N_, float><<<blocks, 128, 0, s>>>(                                   \
          q, box, (const float*)W, face_consts<float>(N_), (float*)FS);                    \
  }
  AWE_FACE(2, 1) AWE_FACE(2, 2) AWE_FACE(2, 3) AWE_FACE(3, 1) AWE_FACE(3, 2) AWE_FACE(3, 3)
#undef AWE_FACE
}

void launch_rk_flux(const Geo& q, int prec, const void* FS, int z0, int z1, void* F, cudaStream_t s) {
  launch_flux_points<true>(q, prec, FS, z0, z1, F, s);
}

// ---------------------------------------------------------------------------
// stage combination (FP64)
// ---------------------------------------------------------------------------
// With div = sum_d (dt/dx_d) (F_{d,i+1/2} - F_{d,i-1/2}) = -dt L(U(k)):
//   o.out = [o.init ? o.a0 U(0) : o.out] + o.al U(k) - o.be div
// for up to two outputs; the first is the stage this call completes (its
// state is checked and, on the last stage, enters the CFL reduction).
template <int D, typename T>
__global__ void __launch_bounds__(256) k_rk_update(Geo q, int z0, int z1, const double* __restrict__ U0,
                                                   const double* __restrict__ Uk, const T* __restrict__ F0,
                                                   const T* __restrict__ F1, const T* __restrict__ F2,
                                                   const double* __restrict__ d_dt, RKOut o1, RKOut o2,
                                                   int nout, unsigned long long* smax, int* err) {
  constexpr int NV = D + 2;
  const int nz = D == 3 ? z1 - z0 : 1;
  const long long nact = (long long)q.n[0] * q.n[1] * nz;
  const double dt = *d_dt;
  double lam[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) lam[d] = dt / q.dx[d];
  double idx_[3] = {1.0 / q.dx[0], 1.0 / q.dx[1], 1.0 / q.dx[2]};
  const long long nx = q.n[0], ny = q.n[1];
  const long long n0 = (nx + 1) * ny * nz, n1 = nx * (ny + 1) * nz, n2 = nx * ny * (nz + 1);
  double m = 0.0;
  bool bad = false;
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < nact;
       z += (long long)gridDim.x * blockDim.x) {
    int i = (int)(z % nx);
    long long t = z / nx;
    int j = (int)(t % ny);
    int kk = (int)(t / ny);
    long long g = gidx(q, i, j, D == 3 ? kk + z0 : 0);
    long long f0 = ((long long)kk * ny + j) * (nx + 1) + i;
    long long f1 = ((long long)kk * (ny + 1) + j) * nx + i;
    long long f2 = ((long long)kk * ny + j) * nx + i;
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double div = lam[0] * ((double)F0[v * n0 + f0 + 1] - (double)F0[v * n0 + f0]);
      div += lam[1] * ((double)F1[v * n1 + f1 + nx] - (double)F1[v * n1 + f1]);
      if (D == 3) div += lam[2] * ((double)F2[v * n2 + f2 + nx * ny] - (double)F2[v * n2 + f2]);
      const long long gv = v * q.ntot + g;
      const double uk = Uk[gv];
      double x = o1.init ? o1.a0 * U0[gv] : o1.out[gv];
      x += o1.al * uk - o1.be * div;
      o1.out[gv] = x;
      u[v] = x;
      if (nout > 1) {
        double y = o2.init ? o2.a0 * U0[gv] : o2.out[gv];
        o2.out[gv] = y + (o2.al * uk - o2.be * div);
      }
    }
    bool ok;
    double sg = zone_signal<D>(u, q.gamma, idx_, ok);
    bad = bad || !ok;
    m = fmax(m, sg);
  }
  if (bad) atomicOr(err, 1);
  if (!smax) return;
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wm[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wm[w] = m;
  __syncthreads();
  if (w == 0) {
    m = lane < (int)(blockDim.x >> 5) ? wm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(smax, (unsigned long long)__double_as_longlong(m));
  }
}

void launch_rk_update(const Geo& q, int prec, const double* U0, const double* Uk, const void* F,
                      const double* d_dt, int z0, int z1, const RKOut& o1, const RKOut& o2, int nout,
                      unsigned long long* smax, int* err, cudaStream_t s) {
  long long off[3] = {0, 0, 0};
  long long acc = 0;
  for (int d = 0; d < q.dim; ++d) {
    int E[3];
    face_ext(q, d, z0, z1, E);
    off[d] = acc;
    acc += (long long)E[0] * E[1] * E[2] * q.nv;
  }
  const int nz = q.dim == 3 ? z1 - z0 : 1;
  long long nact = (long long)q.n[0] * q.n[1] * nz;
  int blocks = grid_for(nact, 256, 152LL * 16);
  if (q.dim == 2) {
    if (prec == AWE_FP64) {
      const double* Fd = (const double*)F;
      k_rk_update<2, double><<<blocks, 256, 0, s>>>(q, z0, z1, U0, Uk, Fd + off[0], Fd + off[1], Fd, d_dt,
                                                    o1, o2, nout, smax, err);
    } else {
      const float* Ff = (const float*)F;
      k_rk_update<2, float><<<blocks, 256, 0, s>>>(q, z0, z1, U0, Uk, Ff + off[0], Ff + off[1], Ff, d_dt,
                                                   o1, o2, nout, smax, err);
    }
  } else {
    if (prec == AWE_FP64) {
      const double* Fd = (const double*)F;
      k_rk_update<3, double><<<blocks, 256, 0, s>>>(q, z0, z1, U0, Uk, Fd + off[0], Fd + off[1],
                                                    Fd + off[2], d_dt, o1, o2, nout, smax, err);
    } else {
      const float* Ff = (const float*)F;
      k_rk_update<3, float><<<blocks, 256, 0, s>>>(q, z0, z1, U0, Uk, Ff + off[0], Ff + off[1],
                                                   Ff + off[2], d_dt, o1, o2, nout, smax, err);
    }
  }
}

}  // namespace awe
