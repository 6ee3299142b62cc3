// Host driver of the bit-pattern conversions in csrc/fp_bits.cuh (the same
// inline functions the FP32 form's reconstruction kernels call): reads n
// doubles and n floats (native byte order) from argv[1], writes the n narrowed
// floats, the n widened non-negative floats and the n widened floats to
// argv[2].
#include <stdio.h>
#include <stdlib.h>

#include "fp_bits.cuh"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  long long n = 0;
  if (fread(&n, sizeof(n), 1, f) != 1 || n < 0) return 4;
  double* x = (double*)malloc(n * sizeof(double) + 1);
  float* b = (float*)malloc(n * sizeof(float) + 1);
  float* y = (float*)malloc(n * sizeof(float) + 1);
  double* w = (double*)malloc(n * sizeof(double) + 1);
  double* g2 = (double*)malloc(n * sizeof(double) + 1);
  if (fread(x, sizeof(double), n, f) != (size_t)n || fread(b, sizeof(float), n, f) != (size_t)n) return 5;
  fclose(f);
  for (long long i = 0; i < n; ++i) {
    y[i] = awe::f64_to_f32_rz(x[i]);
    w[i] = awe::nonneg_f32_to_f64(b[i]);
    g2[i] = awe::f32_to_f64(b[i]);
  }
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 6;
  fwrite(y, sizeof(float), n, g);
  fwrite(w, sizeof(double), n, g);
  fwrite(g2, sizeof(double), n, g);
  fclose(g);
  return 0;
}
