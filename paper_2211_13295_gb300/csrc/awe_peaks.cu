// awe_peaks.cu -- FP64/FP32 FMA throughput of the GPU (the ALU roofline
// denominators): register-resident independent FMA chains, 8 per thread,
// timed with CUDA events, best of 5 launches.
#include "awe_internal.cuh"

namespace awe {

template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fma(acc[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += acc[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static double fma_tflops(int sms, int iters) {
  const int blocks = sms * 4, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
  cudaDeviceSynchronize();
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
}

}  // namespace awe

extern "C" int awe_measure_fma_peaks(double* fp64_tflops, double* fp32_tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AWE_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AWE_ERR_CUDA;
  if (fp64_tflops) *fp64_tflops = awe::fma_tflops<double>(sms, 4096);
  if (fp32_tflops) *fp32_tflops = awe::fma_tflops<float>(sms, 65536);
  return cudaGetLastError() == cudaSuccess ? AWE_OK : AWE_ERR_CUDA;
}
