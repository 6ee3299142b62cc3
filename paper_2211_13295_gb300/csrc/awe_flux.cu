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
#include "awe_flux.cuh"

namespace awe {

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


void launch_flux(const Geo& q, int prec, const void* FS, int z0, int z1, void* F, cudaStream_t s) {
  launch_flux_points<false>(q, prec, FS, z0, z1, F, s);
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
