// awe_gate.h -- learned troubled-zone gate (host side of awe_gate.cu)
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "awe_internal.cuh"

namespace awe {

constexpr int kGateHidden = 32;

struct GateState {
  bool ready = false, have_weights = false;
  int nin = 0;
  size_t np = 0;
  float* params = nullptr;           // device, np floats
  unsigned char* raw = nullptr;      // device, ghosted zones
  unsigned char* flags = nullptr;    // device, ghosted zones
  unsigned char* labels = nullptr;   // device, ghosted zones
  float* feat = nullptr;             // device, ghosted zones x nin (allocated on demand)
  unsigned long long* d_count = nullptr;
  long last_flagged = 0, last_total = 0;
};

__host__ __device__ inline int gate_nin(int dim, int order) { return dim * 2 * (2 * (order - 1) + 1); }
__host__ __device__ inline size_t gate_np(int nin) {
  return (size_t)kGateHidden * nin + kGateHidden + (size_t)kGateHidden * kGateHidden + kGateHidden +
         kGateHidden + 1;
}

int gate_init(GateState& st, const Geo& q, cudaStream_t s);
void gate_free(GateState& st);
int gate_set_weights(GateState& st, const Geo& q, const float* host_params, size_t n, cudaStream_t s);
// flags of the current ghosted state (ghost zones must be filled)
const unsigned char* gate_compute_flags(GateState& st, const Geo& q, int prec, const double* U,
                                        cudaStream_t s);
int gate_features_out(GateState& st, const Geo& q, const double* U, float* out, int on_device,
                      cudaStream_t s);
int gate_labels_out(GateState& st, const Geo& q, const double* U, double tau, unsigned char* out,
                    int on_device, cudaStream_t s);
int gate_stats(GateState& st, const Geo& q, long* flagged, long* total, cudaStream_t s);

}  // namespace awe
