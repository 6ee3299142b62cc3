// awe_flux.cuh -- the face-flux kernel shared by the ADER corrector
// (awe_flux.cu) and the Runge-Kutta variant (awe_rk.cu): per face, the
// Gauss average over NP points of the chosen Riemann solver between the
// upper-face states of the zone below and the lower-face states of the zone
// above.  Each translation unit instantiates only the point count it uses.
#pragma once
#include "awe_internal.cuh"

namespace awe {

// faces normal to d of the slab [z0, z1): index f -> (i, j, k) of the zone
// above the face
__host__ __device__ __forceinline__ void face_ext(const Geo& q, int d, int z0, int z1, int* E) {
  E[0] = q.n[0] + (d == 0);
  E[1] = q.n[1] + (d == 1);
  E[2] = (q.dim == 3 ? z1 - z0 : 1) + (d == 2);
}

// The states are read rotated so that the momentum normal to the face is
// component 1 (then the tangential ones in order of their dimension): the
// Riemann solver runs with a compile-time direction and keeps its arrays in
// registers.  rotated_var gives the stored variable of rotated component r.
template <int D>
__host__ __device__ __forceinline__ int rotated_var(int r, int d) {
  if (r == 0 || r == D + 1) return r;
  if (r == 1) return 1 + d;
  if (r == 2) return d == 0 ? 2 : 1;
  return d == 2 ? 2 : 3;  // r == 3 (3D)
}

// Occupancy: the FP32 kernel waits on its loads of the face states (one
// launch reads ~0.3 GB at 256^3), so it takes as many resident warps as its
// registers allow without spilling (HLLC at 8 points: 64 registers, 32 warps
// per SM; 8.0 -> 4.6 ms per 256^3 step against the compiler's 168
// registers); FP64 is bound by its FP64 arithmetic and keeps the default.
template <int D, int N, typename T, int K, int NP>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? (K == 0 ? (NP == 8 ? 8 : 6) : K == 2 ? 4 : K == 3 ? (D == 3 ? 5 : 6) : 6) : 0) k_flux(Geo q, Region box, int d, int z0, int z1,
                                              const T* __restrict__ FS, T* __restrict__ F) {
  constexpr int NV = D + 2, NFQ = NP;
  int E[3];
  face_ext(q, d, z0, z1, E);
  const long long nf = (long long)E[0] * E[1] * E[2];
  const long long nb = box.size();
  const T gamma = (T)q.gamma;
  const T wq = T(1) / T(NFQ);  // tensor Gauss weights (1/2 per 2-point dimension, 1 for 1 point)
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    split3(f, E[0], E[1], i, j, k);
    if (D == 3) k += z0;
    long long rz = box.index(i, j, k);
    long long lz = rz - (d == 0 ? 1 : d == 1 ? box.ext[0] : (long long)box.ext[0] * box.ext[1]);
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
    // (HLLEM's restored waves hold more live values: unrolling all its points
    // spills in FP64)
#pragma unroll (K == 2 ? 2 : NFQ)
    for (int p = 0; p < NFQ; ++p) {
      T UL[NV], UR[NV], Fp[NV];
#pragma unroll
      for (int r = 0; r < NV; ++r) {
        const int v = rotated_var<D>(r, d);
        UL[r] = FS[((((long long)d * 2 + 1) * NFQ + p) * NV + v) * nb + lz];
        UR[r] = FS[((((long long)d * 2 + 0) * NFQ + p) * NV + v) * nb + rz];
      }
      riemann<K, D, T>(UL, UR, 0, gamma, Fp);
#pragma unroll
      for (int r = 0; r < NV; ++r) acc[r] = fma(wq, Fp[r], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < NV; ++r) F[(long long)rotated_var<D>(r, d) * nf + f] = acc[r];
  }
}

template <int D, int N, bool RK>
__host__ __device__ constexpr int kPoints() {
  return RK ? Modes<D, N>::NFQ / Modes<D, N>::NQ : Modes<D, N>::NFQ;
}

inline int grid_for(long long n, int threads, long long cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// Face-flux launches over the slab [z0, z1): NP = the ADER points (face x
// time, Modes::NFQ) or, for the Runge-Kutta variant (RK = true), the face
// points only (NFQ / NQ).
template <bool RK>
void launch_flux_points(const Geo& q, int prec, const void* FS, int z0, int z1, void* F, cudaStream_t s) {
  Region box = region_box(q, z0, z1);
  long long off = 0;
  for (int d = 0; d < q.dim; ++d) {
    int E[3];
    face_ext(q, d, z0, z1, E);
    long long nf = (long long)E[0] * E[1] * E[2];
    int blocks = grid_for(nf, 128, 152LL * 64);
#define AWE_FLUX_K(D_, N_, K_)                                                        \
    if (q.dim == D_ && q.N == N_ && q.riemann == K_) {                                \
      constexpr int np = kPoints<D_, N_, RK>();                                       \
      if (prec == AWE_FP64)                                                           \
        k_flux<D_, N_, double, K_, np><<<blocks, 128, 0, s>>>(                         \
            q, box, d, z0, z1, (const double*)FS, (double*)F + off);                  \
      else                                                                            \
        k_flux<D_, N_, float, K_, np><<<blocks, 128, 0, s>>>(                          \
            q, box, d, z0, z1, (const float*)FS, (float*)F + off);                    \
    }
#define AWE_FLUX(D_, N_) AWE_FLUX_K(D_, N_, 0) AWE_FLUX_K(D_, N_, 1) AWE_FLUX_K(D_, N_, 2) AWE_FLUX_K(D_, N_, 3)
    AWE_FLUX(2, 1) AWE_FLUX(2, 2) AWE_FLUX(2, 3) AWE_FLUX(3, 1) AWE_FLUX(3, 2) AWE_FLUX(3, 3)
#undef AWE_FLUX
#undef AWE_FLUX_K
    off += nf * q.nv;
  }
}

}  // namespace awe
