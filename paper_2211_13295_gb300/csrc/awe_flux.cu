// awe_flux.cu -- the corrector: face-averaged HLLC fluxes (Make_Flux_X/Y/Z,
// Fig. 5) and the conservative FP64 update with the CFL reduction of the
// updated state (Make_dU_dt and Update_U_Timestep, Figs. 6-7).
//
// Face flux: F = sum_q w_q RS(U_L(q), U_R(q)) over the tensor Gauss-Legendre
// points of the face and of the time step (2 per dimension at orders 3 and 4,
// 1 at order 2), RS one of HLLC (default), HLL, HLLEM or Rusanov,
// U_L from the upper-face states of the zone below the face, U_R from the
// lower-face states of the zone above.  Update: U+ = U - sum_d (dt/dx_d)
// (F_{d,i+1/2} - F_{d,i-1/2}), in FP64 for every form.
#include "awe_internal.cuh"

namespace awe {

// faces normal to d of the slab [z0, z1): index f -> (i, j, k) of the zone
// above the face
__host__ __device__ __forceinline__ void face_ext(const Geo& q, int d, int z0, int z1, int* E) {
  E[0] = q.n[0] + (d == 0);
  E[1] = q.n[1] + (d == 1);
  E[2] = (q.dim == 3 ? z1 - z0 : 1) + (d == 2);
}

template <int D, int N, typename T, int K>
__global__ void __launch_bounds__(128) k_flux(Geo q, Region box, int d, int z0, int z1,
                                              const T* __restrict__ FS, T* __restrict__ F) {
  constexpr int NV = D + 2, NFQ = Modes<D, N>::NFQ;
  int E[3];
  face_ext(q, d, z0, z1, E);
  const long long nf = (long long)E[0] * E[1] * E[2];
  const long long nb = box.size();
  const T gamma = (T)q.gamma;
  const T wq = T(1) / T(NFQ);  // tensor Gauss weights (1/2 per 2-point dimension, 1 for 1 point)
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    int i = (int)(f % E[0]);
    long long t = f / E[0];
    int j = (int)(t % E[1]);
    int k = (int)(t / E[1]) + (D == 3 ? z0 : 0);
    long long rz = box.index(i, j, k);
    long long lz = rz - (d == 0 ? 1 : d == 1 ? box.ext[0] : (long long)box.ext[0] * box.ext[1]);
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
#pragma unroll
    for (int p = 0; p < NFQ; ++p) {
      T UL[NV], UR[NV], Fp[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        UL[v] = FS[((((long long)d * 2 + 1) * NFQ + p) * NV + v) * nb + lz];
        UR[v] = FS[((((long long)d * 2 + 0) * NFQ + p) * NV + v) * nb + rz];
      }
      riemann<K, D, T>(UL, UR, d, gamma, Fp);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = fma(wq, Fp[v], acc[v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) F[(long long)v * nf + f] = acc[v];
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_update(Geo q, int z0, int z1, const double* __restrict__ Uold,
                                                const T* __restrict__ F0, const T* __restrict__ F1,
                                                const T* __restrict__ F2, const double* __restrict__ d_dt,
                                                double* __restrict__ Unew, unsigned long long* smax,
                                                int* err) {
  constexpr int NV = D + 2;
  const int nz = D == 3 ? z1 - z0 : 1;
  const long long nact = (long long)q.n[0] * q.n[1] * nz;
  const double dt = *d_dt;
  double lam[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) lam[d] = dt / q.dx[d];
  double idx_[3] = {1.0 / q.dx[0], 1.0 / q.dx[1], 1.0 / q.dx[2]};
  // face-array extents
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
      double acc = lam[0] * ((double)F0[v * n0 + f0 + 1] - (double)F0[v * n0 + f0]);
      acc += lam[1] * ((double)F1[v * n1 + f1 + nx] - (double)F1[v * n1 + f1]);
      if (D == 3) acc += lam[2] * ((double)F2[v * n2 + f2 + nx * ny] - (double)F2[v * n2 + f2]);
      u[v] = Uold[v * q.ntot + g] - acc;
      Unew[v * q.ntot + g] = u[v];
    }
    bool ok;
    double sg = zone_signal<D>(u, q.gamma, idx_, ok);
    bad = bad || !ok;
    m = fmax(m, sg);
  }
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
  if (bad) atomicOr(err, 1);
}

static int grid_for(long long n, int threads, long long cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

void launch_flux(const Geo& q, int prec, const void* FS, int z0, int z1, void* F, cudaStream_t s) {
  Region box = region_box(q, z0, z1);
  long long off = 0;
  for (int d = 0; d < q.dim; ++d) {
    int E[3];
    face_ext(q, d, z0, z1, E);
    long long nf = (long long)E[0] * E[1] * E[2];
    int blocks = grid_for(nf, 128, 152LL * 64);
#define AWE_FLUX_K(D_, N_, K_)                                                                    \
    if (q.dim == D_ && q.N == N_ && q.riemann == K_) {                                            \
      if (prec == AWE_FP64)                                                                       \
        k_flux<D_, N_, double, K_><<<blocks, 128, 0, s>>>(q, box, d, z0, z1, (const double*)FS,    \
                                                          (double*)F + off);                      \
      else                                                                                        \
        k_flux<D_, N_, float, K_><<<blocks, 128, 0, s>>>(q, box, d, z0, z1, (const float*)FS,      \
                                                         (float*)F + off);                        \
    }
#define AWE_FLUX(D_, N_) AWE_FLUX_K(D_, N_, 0) AWE_FLUX_K(D_, N_, 1) AWE_FLUX_K(D_, N_, 2) AWE_FLUX_K(D_, N_, 3)
    AWE_FLUX(2, 1) AWE_FLUX(2, 2) AWE_FLUX(2, 3) AWE_FLUX(3, 1) AWE_FLUX(3, 2) AWE_FLUX(3, 3)
#undef AWE_FLUX
#undef AWE_FLUX_K
    off += nf * q.nv;
  }
}

void launch_update(const Geo& q, int prec, const double* Uold, const void* F, const double* d_dt,
                   int z0, int z1, double* Unew, unsigned long long* smax, int* err,
                   cudaStream_t s) {
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
      k_update<2, double><<<blocks, 256, 0, s>>>(q, z0, z1, Uold, Fd + off[0], Fd + off[1], Fd, d_dt, Unew, smax, err);
    } else {
      const float* Ff = (const float*)F;
      k_update<2, float><<<blocks, 256, 0, s>>>(q, z0, z1, Uold, Ff + off[0], Ff + off[1], Ff, d_dt, Unew, smax, err);
    }
  } else {
    if (prec == AWE_FP64) {
      const double* Fd = (const double*)F;
      k_update<3, double><<<blocks, 256, 0, s>>>(q, z0, z1, Uold, Fd + off[0], Fd + off[1], Fd + off[2], d_dt, Unew, smax, err);
    } else {
      const float* Ff = (const float*)F;
      k_update<3, float><<<blocks, 256, 0, s>>>(q, z0, z1, Uold, Ff + off[0], Ff + off[1], Ff + off[2], d_dt, Unew, smax, err);
    }
  }
}

}  // namespace awe
