// awe_recon.cu -- WENO reconstruction of the conserved variables into modal
// polynomials (the paper's Limiter stage, Fig. 3, at orders 3 and 4).
//
// Pure modes along an axis come from the 1D WENO of the zone means along that
// axis; a mixed mode is the 1D WENO, along the later axis, of the field of an
// already built mode (u_xy = y-slope of u_x, u_xyy = y-curvature of u_x,
// u_xxy = y-slope of u_xx, likewise with z; u_xyz = z-slope of u_xy).  Three
// passes over the grid, each a coalesced stencil sweep (consecutive threads =
// consecutive x), write the mode fields the next pass needs:
//   pass X on RX = [-1,nx] x [-1-N, ny+N] x [z0-1-N, z1+N]: X[a] = recon_x(U)
//   pass Y on RY = [-1,nx] x [-1, ny] x [z0-1-N, z1+N]:    Y[b] = recon_y(U),
//                                                           XY[a][b] = recon_y(X[a])
//   pass Z on the box [-1,nx] x [-1,ny] x [z0-1, z1]:      the c >= 1 modes,
// and the last pass (Y in 2D, Z in 3D) assembles all modes of the box zones.
// Differences from the zone's own value are taken in FP64 for the zone means
// (rounded toward zero to FP32 in the FP32 form, mean_diff) and in T for mode
// fields; the WENO epsilon path is FP64 (see weno1d).
#include "awe_internal.cuh"

namespace awe {

Region region_x(const Geo& q, int z0, int z1) {
  Region r;
  r.lo[0] = -1; r.ext[0] = q.n[0] + 2;
  r.lo[1] = -1 - q.N; r.ext[1] = q.n[1] + 2 + 2 * q.N;
  if (q.dim == 3) { r.lo[2] = z0 - 1 - q.N; r.ext[2] = z1 - z0 + 2 + 2 * q.N; }
  else { r.lo[2] = 0; r.ext[2] = 1; }
  return r;
}
Region region_y(const Geo& q, int z0, int z1) {
  Region r = region_x(q, z0, z1);
  r.lo[1] = -1; r.ext[1] = q.n[1] + 2;
  return r;
}
Region region_box(const Geo& q, int z0, int z1) {
  Region r = region_y(q, z0, z1);
  if (q.dim == 3) { r.lo[2] = z0 - 1; r.ext[2] = z1 - z0 + 2; }
  return r;
}

// position of spatial mode (a,b,c) in the list "c outer, b, a inner, degree <= N"
template <int D, int N> __host__ __device__ constexpr int mode_index(int a, int b, int c) {
  int idx = 0;
  for (int cc = 0; cc < c; ++cc) idx += (N - cc + 1) * (N - cc + 2) / 2;
  for (int bb = 0; bb < b; ++bb) idx += N - c - bb + 1;
  return idx + a;
}
// number of mixed (a>=1, b>=1, a+b<=N) pairs and the index of one
template <int N> __host__ __device__ constexpr int nxy() { return N * (N - 1) / 2; }

// one 1D reconstruction: WENO at orders 3 and 4, the MC limiter at order 2
template <int N, typename T>
__device__ __forceinline__ void recon1d(const T* d, const Geo& q, bool linear, int v, T* out) {
  if constexpr (N == 1) {
    out[0] = mc_slope<T>(d[2], -d[0], v == 0 ? T(2.0) : T(1.5));
  } else if (linear) {
    if constexpr (sizeof(T) == 8) linear1d<N, T>(d, q.lst, out);
    else linear1d<N, T>(d, q.lstf, out);
  } else {
    weno1d<N, T>(d, q.lin, q.linf, q.eps, false, out);
  }
}
template <int N> __host__ __device__ constexpr int xy_index(int a, int b) {
  int idx = 0;
  for (int aa = 1; aa < a; ++aa) idx += N - aa;
  return idx + (b - 1);
}

// difference of two zone means (FP64) in T
template <typename T> __device__ __forceinline__ T mean_diff(double a, double b) {
  if constexpr (sizeof(T) == 8) return a - b;
  else return f64_to_f32_rz(a - b);
}

__device__ __forceinline__ bool use_linear(const unsigned char* flags, const Geo& q, int i, int j,
                                           int k) {
  return flags != nullptr && flags[gidx(q, i, j, k)] == 0;
}

// ---------------------------------------------------------------------------
template <int D, int N, typename T>
__global__ void __launch_bounds__(128) k_recon_x(Geo q, Region rx, const double* __restrict__ U,
                                                 const unsigned char* __restrict__ flags,
                                                 T* __restrict__ X) {
  const long long nr = rx.size();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
       r += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    rx.coords(r, i, j, k);
    const bool lin = use_linear(flags, q, i, j, k);
    const long long c0 = gidx(q, i, j, k);
#pragma unroll
    for (int v = 0; v < D + 2; ++v) {
      const double* u = U + v * q.ntot + c0;
      double u0 = u[0];
      T d[2 * N + 1];
#pragma unroll
      for (int s = -N; s <= N; ++s) d[s + N] = mean_diff<T>(u[s], u0);
      T out[N];
      recon1d<N, T>(d, q, lin, v, out);
#pragma unroll
      for (int a = 0; a < N; ++a) X[((long long)v * N + a) * nr + r] = out[a];
    }
  }
}

// ---------------------------------------------------------------------------
template <int D, int N, typename T>
__global__ void __launch_bounds__(128) k_recon_y(Geo q, Region rx, Region ry, Region box,
                                                 const double* __restrict__ U,
                                                 const unsigned char* __restrict__ flags,
                                                 const T* __restrict__ X, T* __restrict__ Y,
                                                 T* __restrict__ XY, T* __restrict__ W) {
  constexpr int NS = Modes<D, N>::NS;
  constexpr int NXY = nxy<N>();
  const long long nr = ry.size(), nx_ = rx.size(), nb = box.size();
  const long long ystride = q.G[0];
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr;
       r += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    ry.coords(r, i, j, k);
    const bool lin = use_linear(flags, q, i, j, k);
    const long long c0 = gidx(q, i, j, k);
    const long long xr = rx.index(i, j, k);
    const long long xstride = rx.ext[0];
    // in 2D the region is the box: assemble the modes
    const bool last = (D == 2);
    const long long b = last ? box.index(i, j, k) : 0;
#pragma unroll
    for (int v = 0; v < D + 2; ++v) {
      const double* u = U + v * q.ntot + c0;
      double u0 = u[0];
      T d[2 * N + 1];
#pragma unroll
      for (int s = -N; s <= N; ++s) d[s + N] = mean_diff<T>(u[s * ystride], u0);
      T out[N];
      recon1d<N, T>(d, q, lin, v, out);
      if (!last) {
#pragma unroll
        for (int bb = 0; bb < N; ++bb) Y[((long long)v * N + bb) * nr + r] = out[bb];
      } else {
        W[((long long)v * NS + mode_index<D, N>(0, 0, 0)) * nb + b] = (T)u0;
#pragma unroll
        for (int bb = 1; bb <= N; ++bb) W[((long long)v * NS + mode_index<D, N>(0, bb, 0)) * nb + b] = out[bb - 1];
      }
      // mixed (a, b): recon along y of the X[a] field
#pragma unroll
      for (int a = 1; a <= N; ++a) {
        const T* xa = X + ((long long)v * N + (a - 1)) * nx_ + xr;
        T x0 = xa[0];
        if (last) W[((long long)v * NS + mode_index<D, N>(a, 0, 0)) * nb + b] = x0;
        if (a == N) continue;
        T dx_[2 * N + 1];
#pragma unroll
        for (int s = -N; s <= N; ++s) dx_[s + N] = xa[s * xstride] - x0;
        T o2[N];
        recon1d<N, T>(dx_, q, lin, v, o2);
#pragma unroll
        for (int bb = 1; bb <= N - a; ++bb) {
          if (!last) XY[((long long)v * NXY + xy_index<N>(a, bb)) * nr + r] = o2[bb - 1];
          else W[((long long)v * NS + mode_index<D, N>(a, bb, 0)) * nb + b] = o2[bb - 1];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
template <int N, typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 8 : 0) k_recon_z(Geo q, Region rx, Region ry, Region box,
                                                 const double* __restrict__ U,
                                                 const unsigned char* __restrict__ flags,
                                                 const T* __restrict__ X, const T* __restrict__ Y,
                                                 const T* __restrict__ XY, T* __restrict__ W) {
  constexpr int D = 3;
  constexpr int NS = Modes<D, N>::NS;
  constexpr int NXY = nxy<N>();
  const long long nb = box.size(), nx_ = rx.size(), ny_ = ry.size();
  const long long zstride = (long long)q.G[0] * q.G[1];
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nb;
       r += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    box.coords(r, i, j, k);
    const bool lin = use_linear(flags, q, i, j, k);
    const long long c0 = gidx(q, i, j, k);
    const long long xr = rx.index(i, j, k), yr = ry.index(i, j, k);
    const long long xzs = (long long)rx.ext[0] * rx.ext[1], yzs = (long long)ry.ext[0] * ry.ext[1];
    auto Wp = [&](int v, int a, int b_, int c) -> T& {
      return W[((long long)v * NS + mode_index<D, N>(a, b_, c)) * nb + r];
    };
    // one variable at a time: unrolled over the five, the pass held every
    // variable's stencils at once (255 registers and spills at order 4)
#pragma unroll 1
    for (int v = 0; v < D + 2; ++v) {
      // (0,0,c) from the means
      const double* u = U + v * q.ntot + c0;
      double u0 = u[0];
      T d[2 * N + 1];
#pragma unroll
      for (int s = -N; s <= N; ++s) d[s + N] = mean_diff<T>(u[s * zstride], u0);
      T out[N];
      recon1d<N, T>(d, q, lin, v, out);
      Wp(v, 0, 0, 0) = (T)u0;
#pragma unroll
      for (int c = 1; c <= N; ++c) Wp(v, 0, 0, c) = out[c - 1];
      // (a,0,c) from X[a], (0,b,c) from Y[b]
#pragma unroll
      for (int a = 1; a <= N; ++a) {
        const T* xa = X + ((long long)v * N + (a - 1)) * nx_ + xr;
        const T* ya = Y + ((long long)v * N + (a - 1)) * ny_ + yr;
        T x0 = xa[0], y0 = ya[0];
        Wp(v, a, 0, 0) = x0;
        Wp(v, 0, a, 0) = y0;
        if (a == N) continue;
        T dd[2 * N + 1], o2[N];
#pragma unroll
        for (int s = -N; s <= N; ++s) dd[s + N] = xa[s * xzs] - x0;
        recon1d<N, T>(dd, q, lin, v, o2);
#pragma unroll
        for (int c = 1; c <= N - a; ++c) Wp(v, a, 0, c) = o2[c - 1];
#pragma unroll
        for (int s = -N; s <= N; ++s) dd[s + N] = ya[s * yzs] - y0;
        recon1d<N, T>(dd, q, lin, v, o2);
#pragma unroll
        for (int c = 1; c <= N - a; ++c) Wp(v, 0, a, c) = o2[c - 1];
      }
      // (a,b,0) from XY[a][b]; (a,b,c) with c >= 1 from recon_z(XY[a][b])
#pragma unroll
      for (int a = 1; a < N; ++a)
#pragma unroll
        for (int bb = 1; bb <= N - a; ++bb) {
          const T* xy = XY + ((long long)v * NXY + xy_index<N>(a, bb)) * ny_ + yr;
          T x0 = xy[0];
          Wp(v, a, bb, 0) = x0;
          if (a + bb == N) continue;
          T dd[2 * N + 1], o2[N];
#pragma unroll
          for (int s = -N; s <= N; ++s) dd[s + N] = xy[s * yzs] - x0;
          recon1d<N, T>(dd, q, lin, v, o2);
#pragma unroll
          for (int c = 1; c <= N - a - bb; ++c) Wp(v, a, bb, c) = o2[c - 1];
        }
    }
  }
}

// ---------------------------------------------------------------------------
static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = 152LL * 64;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <int D, int N, typename T>
static void recon_impl(const Geo& q, const double* U, const unsigned char* flags, int z0, int z1,
                       T* X, T* Y, T* XY, T* W, cudaStream_t s, cudaEvent_t* ev) {
  Region rx = region_x(q, z0, z1), ry = region_y(q, z0, z1), box = region_box(q, z0, z1);
  const int th = 128;
  k_recon_x<D, N, T><<<grid_for(rx.size(), th), th, 0, s>>>(q, rx, U, flags, X);
  if (ev) cudaEventRecord(ev[0], s);
  k_recon_y<D, N, T><<<grid_for(ry.size(), th), th, 0, s>>>(q, rx, ry, box, U, flags, X, Y, XY, W);
  if (ev) cudaEventRecord(ev[1], s);
  if constexpr (D == 3) {
    k_recon_z<N, T><<<grid_for(box.size(), th), th, 0, s>>>(q, rx, ry, box, U, flags, X, Y, XY, W);
    if (ev) cudaEventRecord(ev[2], s);
  }
}

void launch_recon(const Geo& q, int prec, const double* U, const unsigned char* flags, int z0,
                  int z1, void* X, void* Y, void* XY, void* W, cudaStream_t s, cudaEvent_t* ev) {
#define AWE_RECON(D_, N_)                                                                       \
  if (q.dim == D_ && q.N == N_) {                                                               \
    if (prec == AWE_FP64)                                                                       \
      recon_impl<D_, N_, double>(q, U, flags, z0, z1, (double*)X, (double*)Y, (double*)XY,      \
                                 (double*)W, s, ev);                                            \
    else                                                                                        \
      recon_impl<D_, N_, float>(q, U, flags, z0, z1, (float*)X, (float*)Y, (float*)XY,          \
                                (float*)W, s, ev);                                              \
    return;                                                                                     \
  }
  AWE_RECON(2, 1)
  AWE_RECON(2, 2)
  AWE_RECON(2, 3)
  AWE_RECON(3, 1)
  AWE_RECON(3, 2)
  AWE_RECON(3, 3)
#undef AWE_RECON
}

}  // namespace awe
