// awe_noalloc.cu -- the CFL time step of a caller's state with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc when they need a time step: a runtime
// that plans every device byte ahead of time and forbids allocation while a
// step runs, a component running under a hard device-memory budget shared
// with others, or a caller for which an allocation failure in the middle of a
// time loop is not an acceptable outcome.  awe_cfl_dt_noalloc serves them: it
// reads a state the caller already holds on the device and writes dt into a
// device scalar the caller owns, and the only scratch it uses (one partial
// maximum per thread block) is the file-scope array below, which exists in
// every GPU that loads the library until the process exits.
//
// The scratch array is shared by every call: calls that overlap on the GPU
// (different streams, or different host threads) race on it and must not be
// issued concurrently.  Each call writes every slot it later reads, so nothing
// needs clearing between calls.
#include <cstdio>
#include <string>

#include "awe_internal.cuh"

namespace awe {
void set_global_error(const std::string& msg);  // awe_api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kZonesPerThread = 16;
constexpr long long kZonesPerBlock = (long long)kThreads * kZonesPerThread;  // 4096
constexpr int kMaxPartials = 65536;                                           // 512 KB of scratch
constexpr long long kMaxZones = kZonesPerBlock * kMaxPartials;                // 268,435,456
constexpr int kMaxDevices = 64;

// one partial maximum per block of the first kernel
static __device__ __align__(256) double g_partials[kMaxPartials];

// host-side device addresses of g_partials, one per device (set up on the
// first call on that device)
double* g_partials_addr[kMaxDevices] = {nullptr};

// Signal speed max over the zones [b*4096, (b+1)*4096) of the caller's state
// (conserved variables, [var][z][y][x], active zones, no ghosts); a zone that
// is not physical makes the partial +inf (dt = 0 signals it).
template <int D>
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const double* __restrict__ U, long long nact,
                                                              double gamma, double ix, double iy, double iz,
                                                              double* __restrict__ partials) {
  const double idx_[3] = {ix, iy, iz};
  double m = 0.0;
  bool bad = false;
  const long long base = (long long)blockIdx.x * kZonesPerBlock;
#pragma unroll 4
  for (int k = 0; k < kZonesPerThread; ++k) {
    long long z = base + (long long)k * kThreads + threadIdx.x;
    if (z >= nact) break;
    double u[D + 2];
#pragma unroll
    for (int v = 0; v < D + 2; ++v) u[v] = U[v * nact + z];
    bool ok;
    double s = awe::zone_signal<D>(u, gamma, idx_, ok);
    bad = bad || !ok;
    m = fmax(m, s);
  }
  if (bad) m = __longlong_as_double(0x7ff0000000000000LL);  // +inf
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wm[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wm[w] = m;
  __syncthreads();
  if (w == 0) {
    m = lane < kThreads / 32 ? wm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) partials[blockIdx.x] = m;
  }
}

// dt = cfl / max of the first nb partials (one block)
__global__ void __launch_bounds__(1024) k_noalloc_final(const double* __restrict__ partials, int nb,
                                                        double cfl, double* __restrict__ dt) {
  double m = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, partials[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wm[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wm[w] = m;
  __syncthreads();
  if (w == 0) {
    m = lane < (int)(blockDim.x >> 5) ? wm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) *dt = cfl / m;
  }
}

int fail(int code, const char* msg) {
  awe::set_global_error(msg);
  return code;
}

}  // namespace

extern "C" int awe_cfl_dt_noalloc(const double* U, int dim, const int* n, const double* dx, double gamma,
                                  double cfl, double* dt, void* stream) {
  if (!U || !n || !dx || !dt) return fail(AWE_ERR_ARG, "awe_cfl_dt_noalloc: null argument");
  if (dim != 2 && dim != 3) return fail(AWE_ERR_ARG, "awe_cfl_dt_noalloc: dim must be 2 or 3");
  if (!(gamma > 1.0) || !(cfl > 0.0)) return fail(AWE_ERR_ARG, "awe_cfl_dt_noalloc: need gamma > 1 and cfl > 0");
  long long nact = 1;
  for (int d = 0; d < dim; ++d) {
    if (n[d] < 1 || !(dx[d] > 0.0)) return fail(AWE_ERR_ARG, "awe_cfl_dt_noalloc: bad grid extent or zone size");
    nact *= n[d];
  }
  if (nact > kMaxZones) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "awe_cfl_dt_noalloc: %lld zones exceed the no-allocation limit of %lld zones", nact, kMaxZones);
    return fail(AWE_ERR_ARG, msg);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(AWE_ERR_CUDA, "awe_cfl_dt_noalloc: no usable current device");
  if (!g_partials_addr[dev]) {
    // set-up, once per device, with that device current: the host-side name
    // g_partials is only a stand-in; the kernels need its device address
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_partials);
    if (e != cudaSuccess) {
      std::string m = std::string("awe_cfl_dt_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return fail(AWE_ERR_CUDA, m.c_str());
    }
    g_partials_addr[dev] = p;
  }
  double* partials = g_partials_addr[dev];
  const int nb = (int)((nact + kZonesPerBlock - 1) / kZonesPerBlock);
  cudaStream_t s = (cudaStream_t)stream;
  const double ix = 1.0 / dx[0], iy = 1.0 / dx[1], iz = dim == 3 ? 1.0 / dx[2] : 1.0;
  if (dim == 2)
    k_noalloc_partial<2><<<nb, kThreads, 0, s>>>(U, nact, gamma, ix, iy, iz, partials);
  else
    k_noalloc_partial<3><<<nb, kThreads, 0, s>>>(U, nact, gamma, ix, iy, iz, partials);
  k_noalloc_final<<<1, 1024, 0, s>>>(partials, nb, cfl, dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::string m = std::string("awe_cfl_dt_noalloc: launch: ") + cudaGetErrorString(e);
    return fail(AWE_ERR_CUDA, m.c_str());
  }
  return AWE_OK;
}
