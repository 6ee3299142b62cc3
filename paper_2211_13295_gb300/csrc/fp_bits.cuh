// fp_bits.cuh -- conversions between FP64 and FP32 of the FP32 form's
// reconstruction and update as operations on the IEEE 754 bit patterns (binary64: 11
// exponent bits, bias 1023, 52 fraction bits; binary32: 8, 127, 23).  The
// hardware conversion issues on the FP64 pipe at the FP64 rate; these run on
// the integer ALU.  Host and device (the host build serves the tests).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace awe {

__host__ __device__ __forceinline__ unsigned f64_hi(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return (unsigned)(u >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned f64_lo(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return (unsigned)u;
#endif
}
__host__ __device__ __forceinline__ double f64_from(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ float f32_from(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned f32_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  memcpy(&u, &x, 4);
  return u;
#endif
}

// Narrowing with rounding toward zero (an IEEE rounding mode: the top 23 of
// the 52 fraction bits, the exponent rebiased by 1023 - 127 = 896).
// Magnitudes below 2^-126 give a signed zero (the subnormal range is
// dropped), finite ones at or above 2^128 and infinities give infinity, NaN
// gives a NaN.
__host__ __device__ __forceinline__ float f64_to_f32_rz(double x) {
  const unsigned hi = f64_hi(x), lo = f64_lo(x);
  const unsigned ah = hi & 0x7fffffffu;
  const unsigned nan = ah > 0x7ff00000u || (ah == 0x7ff00000u && lo != 0u) ? 0x00400000u : 0u;
  const unsigned m = ah < 0x38100000u ? 0u
                   : ah < 0x47f00000u ? ((ah - 0x38000000u) << 3) | (lo >> 29)
                                      : 0x7f800000u | nan;
  return f32_from((hi & 0x80000000u) | m);
}

// Widening of a non-negative FP32 value (a smoothness indicator): exact for
// normal values; below 2^-126 (zero, subnormals) it gives 0, and infinity or
// NaN give a finite double >= 2^128, whose narrowing is infinity.
__host__ __device__ __forceinline__ double nonneg_f32_to_f64(float b) {
  const unsigned u = f32_bits(b);
  return u < 0x00800000u ? 0.0 : f64_from((u >> 3) + 0x38000000u, u << 29);
}

// Widening of any FP32 value: exact for normal values and zeros; subnormal
// values (below 2^-126 in magnitude) give a signed zero; infinities and NaN
// keep their kind.
__host__ __device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = f32_bits(x), a = u & 0x7fffffffu;
  const bool normal = a >= 0x00800000u && a < 0x7f800000u;
  const unsigned hi = normal ? (a >> 3) + 0x38000000u
                    : a < 0x00800000u ? 0u
                                      : 0x7ff00000u | (a > 0x7f800000u ? 0x00080000u : 0u);
  return f64_from((u & 0x80000000u) | hi, normal ? u << 29 : 0u);
}

}  // namespace awe
