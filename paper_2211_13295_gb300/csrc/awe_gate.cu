// awe_gate.cu -- the learned troubled-zone gate: stencil features, a 2x32
// ReLU MLP whose logit decides linear (smooth) vs full WENO reconstruction,
// labels produced by the method itself (deviation of the WENO nonlinear
// weights from the linear weights), and deterministic on-device training
// (forward, backward and Adam with fixed-order reductions, no float atomics).
// The paper has no learned part; this is the project's addition.
//
// The gate decision must come out identical on every implementation, so the
// features are computed with explicitly rounded FP64 operations (no
// contraction) and the MLP runs in FP32 with one fused multiply-add per input
// in index order, accumulator started at the bias.
#include <cstdint>
#include <vector>

#include "awe_gate.h"

namespace awe {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// zone (gi,gj,gk) of the ghosted grid -> nin features; false when the
// stencil does not fit.  For each direction and for rho and E: the 2N
// differences across the stencil over their largest magnitude (the stencil's
// shape), then that magnitude over |f(i)| + 1e-12, times 100, squashed by
// x/(1+x).  Explicitly rounded FP64 operations in a fixed order.
template <int D, int N>
__device__ __forceinline__ bool zone_features(const Geo& q, const double* U, int gi, int gj, int gk,
                                              float* f) {
  const int G[3] = {q.G[0], q.G[1], q.G[2]};
  const int idx[3] = {gi, gj, gk};
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (idx[d] < N || idx[d] > G[d] - 1 - N) return false;
  const long long z = ((long long)gk * G[1] + gj) * G[0] + gi;
  const long long stride[3] = {1, G[0], (long long)G[0] * G[1]};
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int qty = 0; qty < 2; ++qty) {
      const double* u = U + (qty == 0 ? 0 : (long long)(q.nv - 1) * q.ntot) + z;
      double vals[2 * N + 1], del[2 * N];
#pragma unroll
      for (int s = -N; s <= N; ++s) vals[N + s] = u[s * stride[d]];
      double sc = 0.0;
#pragma unroll
      for (int t = 0; t < 2 * N; ++t) {
        del[t] = __dsub_rn(vals[t + 1], vals[t]);
        sc = fmax(sc, fabs(del[t]));
      }
      // divisions, scaling and squashing in FP32, each rounded once
      float* o = f + (d * 2 + qty) * (2 * N + 1);
      const float scf = __double2float_rn(sc);
#pragma unroll
      for (int t = 0; t < 2 * N; ++t) o[t] = scf > 0.0f ? __fdiv_rn(__double2float_rn(del[t]), scf) : 0.0f;
      const float den = __fadd_rn(__double2float_rn(fabs(vals[N])), 1e-12f);
      const float x = __fmul_rn(100.0f, __fdiv_rn(scf, den));
      o[2 * N] = __fdiv_rn(x, __fadd_rn(1.0f, x));
    }
  return true;
}

// FP32 MLP forward in the decision order; params in shared memory
template <int NIN>
__device__ __forceinline__ float mlp_logit(const float* P, const float* x) {
  constexpr int H = kGateHidden;
  const float* W1 = P;
  const float* b1 = W1 + H * NIN;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float* b3 = w3 + H;
  float h1[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    float a = b1[j];
#pragma unroll
    for (int i = 0; i < NIN; ++i) a = __fmaf_rn(W1[j * NIN + i], x[i], a);
    h1[j] = a > 0.0f ? a : 0.0f;
  }
  float o = b3[0];
#pragma unroll 4
  for (int k = 0; k < H; ++k) {
    float a = b2[k];
#pragma unroll
    for (int j = 0; j < H; ++j) a = __fmaf_rn(W2[k * H + j], h1[j], a);
    float h2 = a > 0.0f ? a : 0.0f;
    o = __fmaf_rn(w3[k], h2, o);
  }
  return o;
}

template <int D, int N>
__global__ void __launch_bounds__(128) k_gate_raw(Geo q, const double* __restrict__ U,
                                                  const float* __restrict__ params, int np,
                                                  unsigned char* __restrict__ raw) {
  constexpr int NIN = D * 2 * (2 * N + 1);
  extern __shared__ float sP[];
  for (int i = threadIdx.x; i < np; i += blockDim.x) sP[i] = params[i];
  __syncthreads();
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < q.ntot;
       z += (long long)gridDim.x * blockDim.x) {
    int gi = (int)(z % q.G[0]);
    long long t = z / q.G[0];
    int gj = (int)(t % q.G[1]);
    int gk = (int)(t / q.G[1]);
    float f[NIN];
    if (!zone_features<D, N>(q, U, gi, gj, gk, f)) {
      raw[z] = 1;
      continue;
    }
    raw[z] = mlp_logit<NIN>(sP, f) > 0.0f ? 1 : 0;
  }
}

__global__ void k_gate_dilate(Geo q, const unsigned char* __restrict__ raw,
                              unsigned char* __restrict__ flags) {
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < q.ntot;
       z += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    idx[0] = (int)(z % q.G[0]);
    long long t = z / q.G[0];
    idx[1] = (int)(t % q.G[1]);
    idx[2] = (int)(t / q.G[1]);
    const long long stride[3] = {1, q.G[0], (long long)q.G[0] * q.G[1]};
    unsigned char f = raw[z];
    for (int d = 0; d < q.dim; ++d) {
      if (idx[d] > 0) f |= raw[z - stride[d]];
      if (idx[d] < q.G[d] - 1) f |= raw[z + stride[d]];
    }
    flags[z] = f;
  }
}

template <int D, int N>
__global__ void k_gate_features(Geo q, const double* __restrict__ U, float* __restrict__ out) {
  constexpr int NIN = D * 2 * (2 * N + 1);
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < q.ntot;
       z += (long long)gridDim.x * blockDim.x) {
    int gi = (int)(z % q.G[0]);
    long long t = z / q.G[0];
    int gj = (int)(t % q.G[1]);
    int gk = (int)(t / q.G[1]);
    float f[NIN];
    if (!zone_features<D, N>(q, U, gi, gj, gk, f)) {
#pragma unroll
      for (int i = 0; i < NIN; ++i) f[i] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < NIN; ++i) out[z * NIN + i] = f[i];
  }
}

// labels: max over directions, rho and E, candidates of |omega_k - lin_k| > tau
template <int D, int N>
__global__ void k_gate_labels(Geo q, const double* __restrict__ U, double tau,
                              unsigned char* __restrict__ lab) {
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < q.ntot;
       z += (long long)gridDim.x * blockDim.x) {
    int idx[3];
    idx[0] = (int)(z % q.G[0]);
    long long t = z / q.G[0];
    idx[1] = (int)(t % q.G[1]);
    idx[2] = (int)(t / q.G[1]);
    bool fits = true;
#pragma unroll
    for (int d = 0; d < D; ++d) fits = fits && idx[d] >= N && idx[d] <= q.G[d] - 1 - N;
    if (!fits) {
      lab[z] = 255;
      continue;
    }
    const long long stride[3] = {1, q.G[0], (long long)q.G[0] * q.G[1]};
    int l = 0;
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int vv = 0; vv < 2; ++vv) {
        const double* u = U + (vv ? (q.nv - 1) : 0) * q.ntot + z;
        double d_[2 * N + 1];
#pragma unroll
        for (int s = -N; s <= N; ++s) d_[s + N] = u[s * stride[d]] - u[0];
        double c[N + 1][N];
        weno_candidates<N, double>(d_, c);
        double beta[N + 1], om[N + 1];
#pragma unroll
        for (int k = 0; k <= N; ++k) beta[k] = weno_beta<N, double>(c[k]);
        weno_weights<N>(beta, q.lin, q.eps, om);
#pragma unroll
        for (int k = 0; k <= N; ++k) l |= fabs(om[k] - q.lin[k]) > tau;
      }
    lab[z] = (unsigned char)l;
  }
}

__global__ void k_count_box(Geo q, const unsigned char* __restrict__ flags, unsigned long long* cnt) {
  // box zones: active-relative [-1, n_d] in each active dimension
  int B[3] = {q.n[0] + 2, q.n[1] + 2, q.dim == 3 ? q.n[2] + 2 : 1};
  long long nb = (long long)B[0] * B[1] * B[2];
  unsigned long long c = 0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nb;
       r += (long long)gridDim.x * blockDim.x) {
    int i = (int)(r % B[0]) - 1;
    long long t = r / B[0];
    int j = (int)(t % B[1]) - 1;
    int k = q.dim == 3 ? (int)(t / B[1]) - 1 : 0;
    c += flags[gidx(q, i, j, k)] ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(cnt, c);
}

static int blocks_for(long long n, int th) {
  long long b = (n + th - 1) / th;
  return (int)(b > 152LL * 32 ? 152LL * 32 : (b < 1 ? 1 : b));
}

int gate_init(GateState& st, const Geo& q, cudaStream_t s) {
  if (st.ready) return AWE_OK;
  st.nin = gate_nin(q.dim, q.N + 1);
  st.np = gate_np(st.nin);
  if (cudaMalloc(&st.params, st.np * sizeof(float)) != cudaSuccess) return AWE_ERR_OOM;
  if (cudaMalloc(&st.raw, q.ntot) != cudaSuccess) return AWE_ERR_OOM;
  if (cudaMalloc(&st.flags, q.ntot) != cudaSuccess) return AWE_ERR_OOM;
  if (cudaMalloc(&st.labels, q.ntot) != cudaSuccess) return AWE_ERR_OOM;
  if (cudaMalloc(&st.d_count, sizeof(unsigned long long)) != cudaSuccess) return AWE_ERR_OOM;
  st.ready = true;
  (void)s;
  return AWE_OK;
}

void gate_free(GateState& st) {
  void* p[] = {st.params, st.raw, st.flags, st.labels, st.feat, st.d_count};
  for (void* x : p)
    if (x) cudaFree(x);
  st = GateState();
}

int gate_set_weights(GateState& st, const Geo& q, const float* host_params, size_t n, cudaStream_t s) {
  if (n != st.np) return AWE_ERR_ARG;
  if (cudaMemcpyAsync(st.params, host_params, n * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return AWE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return AWE_ERR_CUDA;
  st.have_weights = true;
  (void)q;
  return AWE_OK;
}

const unsigned char* gate_compute_flags(GateState& st, const Geo& q, int prec, const double* U,
                                        cudaStream_t s) {
  (void)prec;
  int th = 128;
  int bl = blocks_for(q.ntot, th);
  size_t sm = st.np * sizeof(float);
  if (q.dim == 2 && q.N == 2) k_gate_raw<2, 2><<<bl, th, sm, s>>>(q, U, st.params, (int)st.np, st.raw);
  if (q.dim == 2 && q.N == 3) k_gate_raw<2, 3><<<bl, th, sm, s>>>(q, U, st.params, (int)st.np, st.raw);
  if (q.dim == 3 && q.N == 2) k_gate_raw<3, 2><<<bl, th, sm, s>>>(q, U, st.params, (int)st.np, st.raw);
  if (q.dim == 3 && q.N == 3) k_gate_raw<3, 3><<<bl, th, sm, s>>>(q, U, st.params, (int)st.np, st.raw);
  k_gate_dilate<<<bl, th, 0, s>>>(q, st.raw, st.flags);
  cudaMemsetAsync(st.d_count, 0, sizeof(unsigned long long), s);
  k_count_box<<<blocks_for(q.ntot, 256), 256, 0, s>>>(q, st.flags, st.d_count);
  return st.flags;
}

int gate_features_out(GateState& st, const Geo& q, const double* U, float* out, int on_device,
                      cudaStream_t s) {
  float* dst = out;
  size_t bytes = (size_t)q.ntot * st.nin * sizeof(float);
  if (!on_device) {
    if (!st.feat && cudaMalloc(&st.feat, bytes) != cudaSuccess) return AWE_ERR_OOM;
    dst = st.feat;
  }
  int bl = blocks_for(q.ntot, 128);
  if (q.dim == 2 && q.N == 2) k_gate_features<2, 2><<<bl, 128, 0, s>>>(q, U, dst);
  if (q.dim == 2 && q.N == 3) k_gate_features<2, 3><<<bl, 128, 0, s>>>(q, U, dst);
  if (q.dim == 3 && q.N == 2) k_gate_features<3, 2><<<bl, 128, 0, s>>>(q, U, dst);
  if (q.dim == 3 && q.N == 3) k_gate_features<3, 3><<<bl, 128, 0, s>>>(q, U, dst);
  if (!on_device && cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return AWE_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? AWE_OK : AWE_ERR_CUDA;
}

int gate_labels_out(GateState& st, const Geo& q, const double* U, double tau, unsigned char* out,
                    int on_device, cudaStream_t s) {
  unsigned char* dst = on_device ? out : st.labels;
  int bl = blocks_for(q.ntot, 128);
  if (q.dim == 2 && q.N == 2) k_gate_labels<2, 2><<<bl, 128, 0, s>>>(q, U, tau, dst);
  if (q.dim == 2 && q.N == 3) k_gate_labels<2, 3><<<bl, 128, 0, s>>>(q, U, tau, dst);
  if (q.dim == 3 && q.N == 2) k_gate_labels<3, 2><<<bl, 128, 0, s>>>(q, U, tau, dst);
  if (q.dim == 3 && q.N == 3) k_gate_labels<3, 3><<<bl, 128, 0, s>>>(q, U, tau, dst);
  if (!on_device && cudaMemcpyAsync(out, dst, q.ntot, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return AWE_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? AWE_OK : AWE_ERR_CUDA;
}

int gate_stats(GateState& st, const Geo& q, long* flagged, long* total, cudaStream_t s) {
  if (!st.ready) return AWE_ERR_STATE;
  unsigned long long c = 0;
  if (cudaMemcpyAsync(&c, st.d_count, sizeof(c), cudaMemcpyDeviceToHost, s) != cudaSuccess) return AWE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return AWE_ERR_CUDA;
  if (flagged) *flagged = (long)c;
  if (total) *total = (long)(q.n[0] + 2) * (q.n[1] + 2) * (q.dim == 3 ? q.n[2] + 2 : 1);
  return AWE_OK;
}

// ---------------------------------------------------------------------------
// MLP training: per-block forward/backward over a chunk of rows held in shared
// memory, parameter gradients summed over the chunk's rows in index order,
// block partials summed in block order by the optimiser kernel.
// ---------------------------------------------------------------------------
constexpr int kRowsPerBlock = 64;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// rows of the batch: sampled = 1 -> drawn from (seed, step, i); 0 -> row i
__device__ __forceinline__ long batch_row(int sampled, unsigned long long seed, long step, long i, long rows) {
  if (!sampled) return i;
  unsigned long long h = splitmix64(seed ^ splitmix64((unsigned long long)step * 0x100000001B3ull + (unsigned long long)i));
  return (long)(h % (unsigned long long)rows);
}

// partial gradient of one block of rows (mean over the whole batch B)
__global__ void k_mlp_grad(int nin, const float* __restrict__ P, const float* __restrict__ X,
                           const float* __restrict__ Y, long rows, long B, int sampled,
                           unsigned long long seed, long step, float* __restrict__ part,
                           float* __restrict__ loss_part) {
  constexpr int H = kGateHidden;
  extern __shared__ float sm[];
  float* sx = sm;                             // [R][nin]
  float* sh1 = sx + kRowsPerBlock * nin;      // [R][H]
  float* sh2 = sh1 + kRowsPerBlock * H;       // [R][H]
  float* sd1 = sh2 + kRowsPerBlock * H;       // [R][H]
  float* sd2 = sd1 + kRowsPerBlock * H;       // [R][H]
  float* sdz = sd2 + kRowsPerBlock * H;       // [R]
  float* sl = sdz + kRowsPerBlock;            // [R]
  const size_t np = gate_np(nin);
  const float* W1 = P;
  const float* b1 = W1 + H * nin;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float* b3 = w3 + H;
  const long r0 = (long)blockIdx.x * kRowsPerBlock;
  const int nr = (int)((B - r0) < kRowsPerBlock ? (B - r0) : kRowsPerBlock);
  // load rows
  for (int t = threadIdx.x; t < nr * nin; t += blockDim.x) {
    int rr = t / nin, i = t % nin;
    long row = batch_row(sampled, seed, step, r0 + rr, rows);
    sx[t] = X[row * nin + i];
  }
  __syncthreads();
  // forward/backward, one thread per row
  for (int rr = threadIdx.x; rr < nr; rr += blockDim.x) {
    const float* x = sx + rr * nin;
    float a1[H], h1[H], a2[H], h2[H];
    for (int j = 0; j < H; ++j) {
      float a = b1[j];
      for (int i = 0; i < nin; ++i) a = fmaf(W1[j * nin + i], x[i], a);
      a1[j] = a;
      h1[j] = a > 0.f ? a : 0.f;
    }
    float z = b3[0];
    for (int k = 0; k < H; ++k) {
      float a = b2[k];
      for (int j = 0; j < H; ++j) a = fmaf(W2[k * H + j], h1[j], a);
      a2[k] = a;
      h2[k] = a > 0.f ? a : 0.f;
      z = fmaf(w3[k], h2[k], z);
    }
    long row = batch_row(sampled, seed, step, r0 + rr, rows);
    float y = Y[row];
    float lz = fmaxf(z, 0.f) - y * z + log1pf(expf(-fabsf(z)));
    float dz = (1.f / (1.f + expf(-z)) - y) / (float)B;
    float d2[H];
    for (int k = 0; k < H; ++k) d2[k] = a2[k] > 0.f ? dz * w3[k] : 0.f;
    for (int j = 0; j < H; ++j) {
      float s = 0.f;
      for (int k = 0; k < H; ++k) s = fmaf(d2[k], W2[k * H + j], s);
      sd1[rr * H + j] = a1[j] > 0.f ? s : 0.f;
      sh1[rr * H + j] = h1[j];
    }
    for (int k = 0; k < H; ++k) {
      sd2[rr * H + k] = d2[k];
      sh2[rr * H + k] = h2[k];
    }
    sdz[rr] = dz;
    sl[rr] = lz;
  }
  __syncthreads();
  // parameter gradients: each thread owns parameters, sums rows in order
  for (size_t pidx = threadIdx.x; pidx < np; pidx += blockDim.x) {
    float acc = 0.f;
    size_t o = pidx;
    if (o < (size_t)H * nin) {
      int j = (int)(o / nin), i = (int)(o % nin);
      for (int rr = 0; rr < nr; ++rr) acc = fmaf(sd1[rr * H + j], sx[rr * nin + i], acc);
    } else if ((o -= (size_t)H * nin) < H) {
      for (int rr = 0; rr < nr; ++rr) acc += sd1[rr * H + o];
    } else if ((o -= H) < (size_t)H * H) {
      int k = (int)(o / H), j = (int)(o % H);
      for (int rr = 0; rr < nr; ++rr) acc = fmaf(sd2[rr * H + k], sh1[rr * H + j], acc);
    } else if ((o -= (size_t)H * H) < H) {
      for (int rr = 0; rr < nr; ++rr) acc += sd2[rr * H + o];
    } else if ((o -= H) < H) {
      for (int rr = 0; rr < nr; ++rr) acc = fmaf(sdz[rr], sh2[rr * H + o], acc);
    } else {
      for (int rr = 0; rr < nr; ++rr) acc += sdz[rr];
    }
    part[(size_t)blockIdx.x * np + pidx] = acc;
  }
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int rr = 0; rr < nr; ++rr) l += sl[rr];
    loss_part[blockIdx.x] = l;
  }
}

// sum block partials in block order; then Adam (or plain gradient output)
__global__ void k_mlp_reduce_adam(int np, int nblocks, const float* __restrict__ part,
                                  const float* __restrict__ loss_part, long B, float* __restrict__ P,
                                  float* __restrict__ m, float* __restrict__ v, float lr, long t,
                                  float* __restrict__ grad_out, float* __restrict__ loss_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    float g = 0.f;
    for (int b = 0; b < nblocks; ++b) g += part[(size_t)b * np + i];
    if (grad_out) grad_out[i] = g;
    if (m) {
      const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
      float mi = b1 * m[i] + (1.f - b1) * g;
      float vi = b2 * v[i] + (1.f - b2) * g * g;
      m[i] = mi;
      v[i] = vi;
      float mh = mi / (1.f - powf(b1, (float)t));
      float vh = vi / (1.f - powf(b2, (float)t));
      P[i] -= lr * mh / (sqrtf(vh) + eps);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss_out) {
    float l = 0.f;
    for (int b = 0; b < nblocks; ++b) l += loss_part[b];
    *loss_out = l / (float)B;
  }
}

__global__ void k_mlp_forward(int nin, const float* __restrict__ P, const float* __restrict__ X, long B,
                              float* __restrict__ z) {
  constexpr int H = kGateHidden;
  const float* W1 = P;
  const float* b1 = W1 + H * nin;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* w3 = b2 + H;
  const float* b3 = w3 + H;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < B; r += (long)gridDim.x * blockDim.x) {
    const float* x = X + r * nin;
    float h1[H];
    for (int j = 0; j < H; ++j) {
      float a = b1[j];
      for (int i = 0; i < nin; ++i) a = __fmaf_rn(W1[j * nin + i], x[i], a);
      h1[j] = a > 0.f ? a : 0.f;
    }
    float o = b3[0];
    for (int k = 0; k < H; ++k) {
      float a = b2[k];
      for (int j = 0; j < H; ++j) a = __fmaf_rn(W2[k * H + j], h1[j], a);
      float h2 = a > 0.f ? a : 0.f;
      o = __fmaf_rn(w3[k], h2, o);
    }
    z[r] = o;
  }
}

static size_t grad_smem(int nin) {
  return sizeof(float) * ((size_t)kRowsPerBlock * nin + 4 * (size_t)kRowsPerBlock * kGateHidden + 2 * kRowsPerBlock);
}

}  // namespace awe

using namespace awe;

extern "C" {

int awe_gate_dims(int dim, int order, int* nin, size_t* nparams) {
  if ((dim != 2 && dim != 3) || (order != 3 && order != 4)) return AWE_ERR_ARG;
  int n = gate_nin(dim, order);
  if (nin) *nin = n;
  if (nparams) *nparams = gate_np(n);
  return AWE_OK;
}

static int mlp_grad_step(int nin, float* params, float* m, float* v, const float* X, const float* y,
                         long rows, long B, int sampled, unsigned long long seed, long step, float lr,
                         float* grad_out, float* loss_out, cudaStream_t s, float* part, float* lpart) {
  int nblocks = (int)((B + kRowsPerBlock - 1) / kRowsPerBlock);
  size_t np = gate_np(nin);
  k_mlp_grad<<<nblocks, 128, grad_smem(nin), s>>>(nin, params, X, y, rows, B, sampled, seed, step, part, lpart);
  k_mlp_reduce_adam<<<(int)((np + 255) / 256), 256, 0, s>>>((int)np, nblocks, part, lpart, B, params, m, v, lr,
                                                            step + 1, grad_out, loss_out);
  return cudaGetLastError() == cudaSuccess ? AWE_OK : AWE_ERR_CUDA;
}

int awe_mlp_train(int nin, float* params, float* m, float* v, const float* X, const float* y, long rows,
                  int batch, int steps, long step0, float lr, unsigned long long seed, float* loss_out,
                  void* stream) {
  if (nin <= 0 || nin > 64 || !params || !m || !v || !X || !y || rows <= 0 || batch <= 0 || steps < 0)
    return AWE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  size_t np = gate_np(nin);
  int nblocks = (batch + kRowsPerBlock - 1) / kRowsPerBlock;
  float *part = nullptr, *lpart = nullptr;
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem(64)) != cudaSuccess)
    return AWE_ERR_CUDA;
  if (cudaMallocAsync((void**)&part, sizeof(float) * np * nblocks, s) != cudaSuccess) return AWE_ERR_OOM;
  if (cudaMallocAsync((void**)&lpart, sizeof(float) * nblocks, s) != cudaSuccess) return AWE_ERR_OOM;
  int rc = AWE_OK;
  for (int k = 0; k < steps && rc == AWE_OK; ++k)
    rc = mlp_grad_step(nin, params, m, v, X, y, rows, batch, 1, seed, step0 + k, lr, nullptr,
                       loss_out ? loss_out + k : nullptr, s, part, lpart);
  cudaFreeAsync(part, s);
  cudaFreeAsync(lpart, s);
  return rc;
}

int awe_mlp_loss_grad(int nin, const float* params, const float* X, const float* y, long B, float* grad,
                      float* loss, void* stream) {
  if (nin <= 0 || nin > 64 || !params || !X || !y || B <= 0 || !grad) return AWE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  size_t np = gate_np(nin);
  int nblocks = (int)((B + kRowsPerBlock - 1) / kRowsPerBlock);
  float *part = nullptr, *lpart = nullptr;
  if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem(64)) != cudaSuccess)
    return AWE_ERR_CUDA;
  if (cudaMallocAsync((void**)&part, sizeof(float) * np * nblocks, s) != cudaSuccess) return AWE_ERR_OOM;
  if (cudaMallocAsync((void**)&lpart, sizeof(float) * nblocks, s) != cudaSuccess) return AWE_ERR_OOM;
  int rc = mlp_grad_step(nin, const_cast<float*>(params), nullptr, nullptr, X, y, B, B, 0, 0, 0, 0.f, grad,
                         loss, s, part, lpart);
  cudaFreeAsync(part, s);
  cudaFreeAsync(lpart, s);
  return rc;
}

int awe_mlp_forward(int nin, const float* params, const float* X, long B, float* z, void* stream) {
  if (nin <= 0 || !params || !X || !z || B <= 0) return AWE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  long bl = (B + 127) / 128;
  k_mlp_forward<<<(int)(bl > 152 * 16 ? 152 * 16 : bl), 128, 0, s>>>(nin, params, X, B, z);
  return cudaGetLastError() == cudaSuccess ? AWE_OK : AWE_ERR_CUDA;
}

}  // extern "C"
