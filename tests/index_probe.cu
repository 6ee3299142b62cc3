// Host driver of the index decomposition split3 (csrc/awe_internal.cuh, the
// same inline function the kernels call): reads n (r, e0, e1) triples
// (int64, int32, int32; native byte order) from argv[1], writes n (i, j, k)
// int32 triples to argv[2].
#include <stdio.h>
#include <stdlib.h>

#include "awe_internal.cuh"

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  long long n = 0;
  if (fread(&n, sizeof(n), 1, f) != 1 || n < 0) return 4;
  long long* r = (long long*)malloc(n * sizeof(long long) + 1);
  int* e = (int*)malloc(2 * n * sizeof(int) + 1);
  int* out = (int*)malloc(3 * n * sizeof(int) + 1);
  if (fread(r, sizeof(long long), n, f) != (size_t)n || fread(e, sizeof(int), 2 * n, f) != (size_t)(2 * n)) return 5;
  fclose(f);
  for (long long t = 0; t < n; ++t) awe::split3(r[t], e[2 * t], e[2 * t + 1], out[3 * t], out[3 * t + 1], out[3 * t + 2]);
  FILE* g = fopen(argv[2], "wb");
  if (!g) return 6;
  fwrite(out, sizeof(int), 3 * n, g);
  fclose(g);
  return 0;
}
