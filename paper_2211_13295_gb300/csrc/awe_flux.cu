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
    int i, j, kk;
    split3(z, (int)nx, (int)ny, i, j, kk);
    long long g = gidx(q, i, j, D == 3 ? kk + z0 : 0);
    long long f0 = ((long long)kk * ny + j) * (nx + 1) + i;
    long long f1 = ((long long)kk * (ny + 1) + j) * nx + i;
    long long f2 = ((long long)kk * ny + j) * nx + i;
    // FP32 fluxes widen exactly by bit operations (f32_to_f64: the hardware
    // conversion issues on the FP64 pipe; a subnormal flux counts as zero on
    // both of its zones, so the update stays conservative)
    auto wd = [](T x) -> double {
      if constexpr (sizeof(T) == 8) return x;
      else return f32_to_f64(x);
    };
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double acc = lam[0] * (wd(F0[v * n0 + f0 + 1]) - wd(F0[v * n0 + f0]));
      acc += lam[1] * (wd(F1[v * n1 + f1 + nx]) - wd(F1[v * n1 + f1]));
      if (D == 3) acc += lam[2] * (wd(F2[v * n2 + f2 + nx * ny]) - wd(F2[v * n2 + f2]));
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


// ---------------------------------------------------------------------------
// A posteriori fallback (awe_config.fallback = 2; not in the paper).  The
// high-order fluxes of every slab are kept in a whole-grid FP64 buffer; after
// the update, passes flag the zones whose new mean is not physical (flags
// accumulate) and update again every flagged zone and every zone sharing a
// face with one, from the old state, with the Riemann flux between the two
// old zone means on each face next to a flagged zone and the kept high-order
// flux elsewhere.  Both zones of a face see the same flux (conservative).
// Across a periodic face the neighbour is the periodic image; other boundary
// faces have no neighbour to flag.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ long long faces_full(const Geo& q, int d) {
  return (long long)(q.n[0] + (d == 0)) * (q.n[1] + (d == 1)) * (q.dim == 3 ? q.n[2] + (d == 2) : 1);
}

template <typename T>
__global__ void k_store_fluxes(Geo q, int z0, int z1, const T* __restrict__ F, double* __restrict__ Ffull) {
  long long offS = 0, offF = 0;
  for (int d = 0; d < q.dim; ++d) {
    int E[3];
    face_ext(q, d, z0, z1, E);
    const long long ns = (long long)E[0] * E[1] * E[2], nf = faces_full(q, d);
    for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < ns * q.nv;
         z += (long long)gridDim.x * blockDim.x) {
      const int v = (int)(z / ns);
      const long long f = z - v * ns;
      const int i = (int)(f % E[0]);
      const long long t = f / E[0];
      const int j = (int)(t % E[1]);
      const int k = (int)(t / E[1]) + (q.dim == 3 ? z0 : 0);
      const long long ff = ((long long)k * E[1] + j) * E[0] + i;
      Ffull[offF + v * nf + ff] = (double)F[offS + v * ns + f];
    }
    offS += ns * q.nv;
    offF += nf * q.nv;
  }
}

template <int D>
__global__ void k_fb_flag(Geo q, const double* __restrict__ U, unsigned char* __restrict__ flags) {
  const long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < nact;
       z += (long long)gridDim.x * blockDim.x) {
    if (flags[z]) continue;
    const int i = (int)(z % q.n[0]);
    const long long t = z / q.n[0];
    const int j = (int)(t % q.n[1]), k = (int)(t / q.n[1]);
    double u[D + 2];
    const long long g = gidx(q, i, j, k);
#pragma unroll
    for (int v = 0; v < D + 2; ++v) u[v] = U[v * q.ntot + g];
    if (!state_physical<D, double>(u, q.gamma - 1.0)) flags[z] = 1;
  }
}

template <int D, int K>
__global__ void k_fb_refit(Geo q, const double* __restrict__ Uold, const double* __restrict__ Ffull,
                           const unsigned char* __restrict__ flags, const double* __restrict__ d_dt,
                           double* __restrict__ Unew) {
  constexpr int NV = D + 2;
  const long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  const double dt = *d_dt;
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < nact;
       z += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    idx[0] = (int)(z % q.n[0]);
    const long long t = z / q.n[0];
    idx[1] = (int)(t % q.n[1]);
    idx[2] = (int)(t / q.n[1]);
    bool nfl[3][2] = {{false, false}, {false, false}, {false, false}};
    bool near = flags[z] != 0;
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        int m[3] = {idx[0], idx[1], idx[2]};
        m[d] += s ? 1 : -1;
        bool have = true;
        if (m[d] < 0 || m[d] >= q.n[d]) {
          have = q.bc[2 * d + s] == AWE_BC_PERIODIC;
          m[d] = (m[d] + q.n[d]) % q.n[d];
        }
        if (have && flags[((long long)m[2] * q.n[1] + m[1]) * q.n[0] + m[0]]) {
          nfl[d][s] = true;
          near = true;
        }
      }
    if (!near) continue;
    const long long g = gidx(q, idx[0], idx[1], idx[2]);
    double U0[NV], acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      U0[v] = Uold[v * q.ntot + g];
      acc[v] = 0.0;
    }
    long long off = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const long long nf = faces_full(q, d);
      const int E0 = q.n[0] + (d == 0), E1 = q.n[1] + (d == 1);
      double Fs[2][NV];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (flags[z] || nfl[d][s]) {
          // first order: the Riemann flux between the two old zone means
          // (the neighbour may be a ghost zone), states rotated so that the
          // normal momentum is component 1
          int m[3] = {idx[0], idx[1], idx[2]};
          m[d] += s ? 1 : -1;
          const long long gn = gidx(q, m[0], m[1], m[2]);
          double UL[NV], UR[NV], Fr[NV];
#pragma unroll
          for (int r = 0; r < NV; ++r) {
            const int v = rotated_var<D>(r, d);
            const double a = U0[v], b = Uold[v * q.ntot + gn];
            UL[r] = s ? a : b;
            UR[r] = s ? b : a;
          }
          riemann<K, D, double>(UL, UR, 0, q.gamma, Fr);
#pragma unroll
          for (int r = 0; r < NV; ++r) Fs[s][rotated_var<D>(r, d)] = Fr[r];
        } else {
          int fi[3] = {idx[0], idx[1], idx[2]};
          fi[d] += s;
          const long long f = ((long long)(D == 3 ? fi[2] : 0) * E1 + fi[1]) * E0 + fi[0];
#pragma unroll
          for (int v = 0; v < NV; ++v) Fs[s][v] = Ffull[off + v * nf + f];
        }
      }
      const double lam = dt / q.dx[d];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += lam * (Fs[1][v] - Fs[0][v]);
      off += nf * NV;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) Unew[v * q.ntot + g] = U0[v] - acc[v];
  }
}

void launch_store_fluxes(const Geo& q, int prec, const void* F, int z0, int z1, double* Ffull, cudaStream_t s) {
  long long ns = 0;
  for (int d = 0; d < q.dim; ++d) {
    int E[3];
    face_ext(q, d, z0, z1, E);
    ns = E[0] * (long long)E[1] * E[2] * q.nv > ns ? E[0] * (long long)E[1] * E[2] * q.nv : ns;
  }
  const int blocks = grid_for(ns, 256, 152LL * 16);
  if (prec == AWE_FP64) k_store_fluxes<double><<<blocks, 256, 0, s>>>(q, z0, z1, (const double*)F, Ffull);
  else k_store_fluxes<float><<<blocks, 256, 0, s>>>(q, z0, z1, (const float*)F, Ffull);
}

void launch_fb_passes(const Geo& q, const double* Uold, double* Unew, const double* Ffull, unsigned char* flags,
                      const double* d_dt, int passes, cudaStream_t s) {
  const long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  const int blocks = grid_for(nact, 256, 152LL * 16);
  cudaMemsetAsync(flags, 0, (size_t)nact, s);
  for (int p = 0; p < passes; ++p) {
    if (q.dim == 2) k_fb_flag<2><<<blocks, 256, 0, s>>>(q, Unew, flags);
    else k_fb_flag<3><<<blocks, 256, 0, s>>>(q, Unew, flags);
#define AWE_FB(D_, K_) \
    if (q.dim == D_ && q.riemann == K_) k_fb_refit<D_, K_><<<blocks, 256, 0, s>>>(q, Uold, Ffull, flags, d_dt, Unew);
    AWE_FB(2, 0) AWE_FB(2, 1) AWE_FB(2, 2) AWE_FB(2, 3) AWE_FB(3, 0) AWE_FB(3, 1) AWE_FB(3, 2) AWE_FB(3, 3)
#undef AWE_FB
  }
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
