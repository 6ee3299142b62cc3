// awe_rk.h -- the Runge-Kutta variant (awe_rk.cu): Shu-Osher tables of the
// SSP schemes, stage outputs and the per-stage launchers.
#pragma once
#include <cuda_runtime.h>

#include "awe_tables.h"

namespace awe {

struct Geo;
constexpr int kRKMax = 5;

// U(i) = sum_{k<i} alpha[i][k] U(k) + beta[i][k] dt L(U(k)); c[i] the stage
// abscissae (U(i) approximates the solution at t + c[i] dt).
struct RKScheme {
  int s;
  double alpha[kRKMax + 1][kRKMax], beta[kRKMax + 1][kRKMax], c[kRKMax + 1];
};
bool rk_scheme(int stages, RKScheme& r);

// One output of a stage combination: out = [init ? a0 U(0) : out] + al U(k) - be div.
struct RKOut {
  double* out;
  double a0, al, be;
  int init;
};

void launch_face_eval(const Geo& q, int prec, const void* W, int z0, int z1, const void* tab,
                      const PTabLayout& L, void* FS, cudaStream_t s);
void launch_rk_flux(const Geo& q, int prec, const void* FS, int z0, int z1, void* F, cudaStream_t s);
void launch_rk_update(const Geo& q, int prec, const double* U0, const double* Uk, const void* F,
                      const double* d_dt, int z0, int z1, const RKOut& o1, const RKOut& o2, int nout,
                      unsigned long long* smax, int* err, cudaStream_t s);

}  // namespace awe
