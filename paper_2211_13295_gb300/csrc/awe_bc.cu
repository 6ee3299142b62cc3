// awe_bc.cu -- ghost zones (Boundary_Conditions, Fig. 1), the CFL
// max-reduction (Eval_Tstep_Ptwise with REDUCTION(MIN:dt_next), Fig. 7) and
// the device-resident time/time-step scalars.
#include "awe_internal.cuh"

namespace awe {

// Ghost zones: BCs applied dimension after dimension (x, then y, then z), so a
// corner ghost is the z-image of the y-image of the x-image.  Resolved here
// from the outermost dimension inwards; reflections accumulate sign flips of
// the normal momentum, a fixed state ends the chain.
__global__ void k_fill_ghosts(Geo q, double* __restrict__ U, const double* __restrict__ d_t,
                              const double* __restrict__ d_dt, double c) {
  const long long total = q.ntot;
  // time of the boundary values: t, or a Runge-Kutta stage's t + c dt
  // (rounded as written: no contraction into an FMA)
  const double t = c != 0.0 ? __dadd_rn(*d_t, __dmul_rn(c, *d_dt)) : *d_t;
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < total;
       z += (long long)gridDim.x * blockDim.x) {
    int gi = (int)(z % q.G[0]);
    long long r = z / q.G[0];
    int gj = (int)(r % q.G[1]);
    int gk = (int)(r / q.G[1]);
    int idx[3] = {gi - q.g, gj - q.g, q.dim == 3 ? gk - q.g : 0};
    bool inside = true;
    for (int d = 0; d < q.dim; ++d) inside = inside && idx[d] >= 0 && idx[d] < q.n[d];
    if (inside) continue;
    double sign[kMaxV];
    for (int v = 0; v < q.nv; ++v) sign[v] = 1.0;
    const double* fixed = nullptr;
    const double xc = q.lo[0] + (idx[0] + 0.5) * q.dx[0];
    bool external = false;
    for (int d = q.dim - 1; d >= 0 && !fixed && !external; --d) {
      if (idx[d] >= 0 && idx[d] < q.n[d]) continue;
      int side = idx[d] < 0 ? 0 : 1;
      int bc = q.bc[2 * d + side];
      if (bc == AWE_BC_DMR_BOTTOM) bc = (xc < 1.0 / 6.0) ? AWE_BC_INFLOW : AWE_BC_REFLECT;
      switch (bc) {
        case AWE_BC_EXCHANGE:
          // a neighbour's plane, written by awe_halo_unpack (only on the
          // outermost dimension, which this loop resolves first)
          external = true;
          break;
        case AWE_BC_PERIODIC: {
          int m = idx[d] % q.n[d];
          idx[d] = m < 0 ? m + q.n[d] : m;
          break;
        }
        case AWE_BC_OUTFLOW:
          idx[d] = side ? q.n[d] - 1 : 0;
          break;
        case AWE_BC_REFLECT:
          idx[d] = side ? 2 * q.n[d] - 1 - idx[d] : -1 - idx[d];
          sign[1 + d] = -sign[1 + d];
          break;
        case AWE_BC_INFLOW:
          fixed = q.inflow[2 * d + side];
          break;
        case AWE_BC_DMR_TOP: {
          double xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / sqrt(3.0);
          fixed = (xc < xs) ? q.inflow[2 * d + side] : q.pre;
          break;
        }
        default:
          fixed = q.pre;
      }
    }
    if (external) continue;
    if (fixed) {
      for (int v = 0; v < q.nv; ++v) U[v * q.ntot + z] = sign[v] * fixed[v];
    } else {
      long long src = gidx(q, idx[0], idx[1], idx[2]);
      for (int v = 0; v < q.nv; ++v) U[v * q.ntot + z] = sign[v] * U[v * q.ntot + src];
    }
  }
}

void launch_fill_ghosts(const Geo& q, double* U, const double* d_t, const double* d_dt, double c,
                        cudaStream_t s) {
  long long total = q.ntot;
  int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_fill_ghosts<<<(int)blocks, threads, 0, s>>>(q, U, d_t, d_dt, c);
}

// Halo planes of the outermost dimension od (z in 3D, y in 2D) for a slab
// decomposition: buffer [var][plane p][inner ghosted extent].  Pack reads the
// active planes p (low side) or n - g + p (high side); unpack writes the ghost
// planes -g + p (low) or n + p (high), in active coordinates.  The ghosted
// index of plane k along od times the inner extent is the offset of its first
// zone, because od is the slowest dimension of the layout.
__global__ void k_halo_pack(Geo q, const double* __restrict__ U, int side, double* __restrict__ buf) {
  const int od = q.dim - 1;
  const long long plane = od == 2 ? (long long)q.G[0] * q.G[1] : (long long)q.G[0];
  const long long per_v = (long long)q.g * plane;
  const long long n = (long long)q.nv * per_v;
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < n;
       z += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(z / per_v);
    const long long rem = z - v * per_v;
    const int p = (int)(rem / plane);
    const long long o = rem - p * plane;
    const int k = (side ? q.n[od] - q.g + p : p) + q.g;  // ghosted index along od
    buf[z] = U[v * q.ntot + k * plane + o];
  }
}
__global__ void k_halo_unpack(Geo q, double* __restrict__ U, int side, const double* __restrict__ buf) {
  const int od = q.dim - 1;
  const long long plane = od == 2 ? (long long)q.G[0] * q.G[1] : (long long)q.G[0];
  const long long per_v = (long long)q.g * plane;
  const long long n = (long long)q.nv * per_v;
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < n;
       z += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(z / per_v);
    const long long rem = z - v * per_v;
    const int p = (int)(rem / plane);
    const long long o = rem - p * plane;
    const int k = side ? q.n[od] + q.g + p : p;  // ghosted index along od
    U[v * q.ntot + k * plane + o] = buf[z];
  }
}
long long halo_count(const Geo& q) {
  const long long plane = q.dim == 3 ? (long long)q.G[0] * q.G[1] : (long long)q.G[0];
  return (long long)q.nv * q.g * plane;
}
void launch_halo(const Geo& q, double* U, int side, double* buf, bool pack, cudaStream_t s) {
  long long blocks = (halo_count(q) + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (pack) k_halo_pack<<<(int)blocks, 256, 0, s>>>(q, U, side, buf);
  else k_halo_unpack<<<(int)blocks, 256, 0, s>>>(q, U, side, buf);
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }
void launch_set_scalar(double* p, double v, cudaStream_t s) { k_set_scalar<<<1, 1, 0, s>>>(p, v); }

// Warp-shuffle max of the per-zone signal speed, then one atomic per block on
// the bit pattern (a positive double orders like its unsigned bits).
template <int D>
__global__ void k_signal_max(Geo q, const double* __restrict__ U, unsigned long long* smax,
                             int* err) {
  const long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  double idx_[3] = {1.0 / q.dx[0], 1.0 / q.dx[1], 1.0 / q.dx[2]};
  double m = 0.0;
  bool bad = false;
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < nact;
       z += (long long)gridDim.x * blockDim.x) {
    int i = (int)(z % q.n[0]);
    long long r = z / q.n[0];
    int j = (int)(r % q.n[1]);
    int k = (int)(r / q.n[1]);
    long long gz = gidx(q, i, j, k);
    double u[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; ++v) u[v] = U[v * q.ntot + gz];
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

void launch_signal_max(const Geo& q, const double* U, unsigned long long* smax, int* err,
                       cudaStream_t s) {
  long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  int threads = 256;
  long long blocks = (nact + threads - 1) / threads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (q.dim == 2) k_signal_max<2><<<(int)blocks, threads, 0, s>>>(q, U, smax, err);
  else k_signal_max<3><<<(int)blocks, threads, 0, s>>>(q, U, smax, err);
}

// dt_next = cfl / smax; optionally t += dt first; smax reset for the next use.
__global__ void k_finalize(double* d_t, double* d_dt, unsigned long long* smax, double cfl,
                           int advance) {
  if (advance) *d_t += *d_dt;
  double m = __longlong_as_double((long long)*smax);
  *d_dt = cfl / m;
  *smax = 0ull;
}
void launch_finalize(const Geo& q, double* d_t, double* d_dt, unsigned long long* smax,
                     int advance, cudaStream_t s) {
  k_finalize<<<1, 1, 0, s>>>(d_t, d_dt, smax, q.cfl, advance);
}

}  // namespace awe
