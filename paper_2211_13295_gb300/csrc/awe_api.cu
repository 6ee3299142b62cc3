// awe_api.cu -- C ABI of libawe.so (include/awe.h): grid lifetime, device
// memory, the step pipeline, per-stage probes and kernel timing.
//
// One step (the loop body of Fig. 1):
//   ghost zones of U_cur                                   (Boundary_Conditions)
//   [gate: features -> MLP -> flags]                        (learned part)
//   for each z-slab [z0, z1):
//     recon X, Y, (Z) -> modes W of the slab box          (Limiter, Fig. 3)
//     predictor -> face quadrature states FS               (Predictor, Fig. 4)
//     HLLC face fluxes F                                    (Make_Flux, Fig. 5)
//     FP64 update U_nxt = U_cur - dt div F, signal max     (Figs. 6-7)
//   t += dt, dt_next = cfl / smax                          (device scalars)
// The state never leaves the device between steps; dt can stay on the
// device as well (awe_step with dt <= 0).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "awe_gate.h"
#include "awe_internal.cuh"
#include "awe_rk.h"
#include "awe_tables.h"

namespace awe {
cudaError_t predict_init(cudaStream_t s);
void launch_predict_tab(const Geo& q, int prec, int picard, const void* W, const double* d_dt,
                        int z0, int z1, const void* tab, const PTabLayout& L, void* FS,
                        cudaStream_t s);
}  // namespace awe

using namespace awe;

namespace {

enum Kind { K_GHOST = 0, K_RX, K_RY, K_RZ, K_PRED, K_FLUX, K_UPD, K_GATE, K_MISC, K_FACE, K_COUNT };
const char* kKindNames[K_COUNT] = {"fill_ghosts", "recon_x", "recon_y", "recon_z", "predictor",
                                   "riemann_flux", "update_cfl", "gate", "misc", "face_eval"};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kinds;  // kind of interval i = (pool[2i], pool[2i+1]) ... stored as pairs
  std::vector<std::pair<int, int>> spans;  // (event index start, event index end)
  std::vector<int> span_kind;
  size_t used = 0;
  long launches[K_COUNT] = {0};
  double ms[K_COUNT] = {0};
};

}  // namespace

struct awe_grid {
  awe_config cfg;
  Geo q;
  cudaStream_t s = nullptr;
  int prec = 0, picard = 0, slab = 0;
  double* U[2] = {nullptr, nullptr};
  int cur = 0;
  double* d_scal = nullptr;  // [0] t, [1] dt, [2] saved dt
  unsigned long long* d_smax = nullptr;
  unsigned long long* d_fb = nullptr;  // zones sent to the positivity fallback
  int* d_err = nullptr;
  void *X = nullptr, *Y = nullptr, *XY = nullptr, *W = nullptr, *FS = nullptr, *F = nullptr;
  double* stage = nullptr;  // state staging [nv][nact]
  double* Urk[2] = {nullptr, nullptr};  // Runge-Kutta stage states (ghosted)
  awe::RKScheme rk;
  int next_stage = 0;       // stage of the current step that runs next (awe_stage)
  // a posteriori fallback (cfg.fallback = 2): whole-grid high-order fluxes,
  // zone flags, and scratch targets of the first update's CFL max and status
  double* Ffb = nullptr;
  unsigned char* fbflag = nullptr;
  unsigned long long* d_smax2 = nullptr;
  int* d_err2 = nullptr;
  double* halo_stage = nullptr;  // host-pointer halo transfers [halo_count]
  bool poison = false;  // AWE_POISON=1 at create: NaN-fill the intermediates before use
  long long szX = 0, szY = 0, szXY = 0, szW = 0, szFS = 0, szF = 0;
  void* ptab = nullptr;
  PTabLayout L;
  size_t bytesT = 8;
  awe::GateState gate;
  std::string err;
  Prof prof;
};

static std::string g_create_error;

namespace awe {
// message for awe_last_error(NULL) from entry points without a handle
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace awe

namespace {

size_t tsize(int prec) { return prec == AWE_FP64 ? sizeof(double) : sizeof(float); }

int fail(awe_grid* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(awe_grid* g, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // a non-sticky error (a rejected argument) must not resurface in a later call
  return fail(g, e == cudaErrorMemoryAllocation ? AWE_ERR_OOM : AWE_ERR_CUDA, m);
}

#define CK(g, call)                                        \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(g, e_, #call); \
  } while (0)

// ---- profiling helpers ------------------------------------------------------
cudaEvent_t prof_event(awe_grid* g) {
  Prof& p = g->prof;
  if (p.used == p.pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    p.pool.push_back(e);
  }
  return p.pool[p.used++];
}
int prof_mark(awe_grid* g) {
  if (!g->prof.on) return -1;
  cudaEvent_t e = prof_event(g);
  cudaEventRecord(e, g->s);
  return (int)g->prof.used - 1;
}
void prof_span(awe_grid* g, int kind, int a, int b) {
  if (!g->prof.on || a < 0 || b < 0) return;
  g->prof.spans.push_back({a, b});
  g->prof.span_kind.push_back(kind);
}
void prof_collect(awe_grid* g) {
  Prof& p = g->prof;
  if (p.spans.empty()) return;
  cudaStreamSynchronize(g->s);
  for (size_t i = 0; i < p.spans.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.pool[p.spans[i].first], p.pool[p.spans[i].second]);
    p.ms[p.span_kind[i]] += ms;
    p.launches[p.span_kind[i]] += 1;
  }
  p.spans.clear();
  p.span_kind.clear();
  p.used = 0;
}

// ---- state layout kernels ----------------------------------------------------
__global__ void k_scatter(Geo q, const double* __restrict__ src, double* __restrict__ U) {
  long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < nact * q.nv;
       z += (long long)gridDim.x * blockDim.x) {
    int v = (int)(z / nact);
    long long a = z % nact;
    int i = (int)(a % q.n[0]);
    long long t = a / q.n[0];
    int j = (int)(t % q.n[1]);
    int k = (int)(t / q.n[1]);
    U[v * q.ntot + gidx(q, i, j, k)] = src[z];
  }
}
__global__ void k_gather(Geo q, const double* __restrict__ U, double* __restrict__ dst) {
  long long nact = (long long)q.n[0] * q.n[1] * q.n[2];
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < nact * q.nv;
       z += (long long)gridDim.x * blockDim.x) {
    int v = (int)(z / nact);
    long long a = z % nact;
    int i = (int)(a % q.n[0]);
    long long t = a / q.n[0];
    int j = (int)(t % q.n[1]);
    int k = (int)(t / q.n[1]);
    dst[z] = U[v * q.ntot + gidx(q, i, j, k)];
  }
}
template <typename T>
__global__ void k_to_double(const T* __restrict__ a, double* __restrict__ b, long long n) {
  for (long long z = blockIdx.x * (long long)blockDim.x + threadIdx.x; z < n;
       z += (long long)gridDim.x * blockDim.x)
    b[z] = (double)a[z];
}

long long nactive(const Geo& q) { return (long long)q.n[0] * q.n[1] * q.n[2]; }

int nslabs(const awe_grid* g) {
  if (g->q.dim == 2) return 1;
  return (g->q.n[2] + g->slab - 1) / g->slab;
}
void slab_range(const awe_grid* g, int sidx, int& z0, int& z1) {
  if (g->q.dim == 2) { z0 = 0; z1 = 1; return; }
  z0 = sidx * g->slab;
  z1 = z0 + g->slab < g->q.n[2] ? z0 + g->slab : g->q.n[2];
}

// sizes of the slab buffers (elements)
struct Sizes { long long X, Y, XY, W, FS, F; };
Sizes buffer_sizes(const Geo& q, int slab) {
  int z1 = q.dim == 3 ? slab : 1;
  Region rx = region_x(q, 0, z1), ry = region_y(q, 0, z1), box = region_box(q, 0, z1);
  int NS = (int)spatial_modes(q.dim, q.N).size();
  int NXY = q.N * (q.N - 1) / 2;
  int nq = (q.N + 2) / 2;
  int NFQ = q.dim == 3 ? nq * nq * nq : nq * nq;
  Sizes s;
  s.X = (long long)q.nv * q.N * rx.size();
  s.Y = q.dim == 3 ? (long long)q.nv * q.N * ry.size() : 1;
  s.XY = q.dim == 3 && NXY > 0 ? (long long)q.nv * NXY * ry.size() : 1;
  s.W = (long long)q.nv * NS * box.size();
  s.FS = (long long)q.dim * 2 * NFQ * q.nv * box.size();
  s.F = 0;
  for (int d = 0; d < q.dim; ++d) {
    long long e = (long long)(q.n[0] + (d == 0)) * (q.n[1] + (d == 1)) * ((q.dim == 3 ? z1 : 1) + (d == 2));
    s.F += e * q.nv;
  }
  return s;
}

// Debug aid (AWE_POISON=1 at awe_create): every intermediate buffer is filled
// with NaN bit patterns before each slab's pipeline, so that a kernel reading
// an element that no earlier stage of the same slab wrote makes the result
// differ (tests compare poisoned and plain steps bit for bit).
void poison_slab_buffers(awe_grid* g) {
  if (!g->poison) return;
  const size_t b = g->bytesT;
  cudaMemsetAsync(g->X, 0xFF, b * g->szX, g->s);
  cudaMemsetAsync(g->Y, 0xFF, b * g->szY, g->s);
  cudaMemsetAsync(g->XY, 0xFF, b * g->szXY, g->s);
  cudaMemsetAsync(g->W, 0xFF, b * g->szW, g->s);
  cudaMemsetAsync(g->FS, 0xFF, b * g->szFS, g->s);
  cudaMemsetAsync(g->F, 0xFF, b * g->szF, g->s);
}

// the pipeline of one slab: recon, predictor, flux, (update)
void run_slab(awe_grid* g, int z0, int z1, bool do_flux, bool do_update, const unsigned char* flags) {
  const Geo& q = g->q;
  poison_slab_buffers(g);
  int m0 = prof_mark(g);
  cudaEvent_t evs[3];
  cudaEvent_t* ev = nullptr;
  int mi[3] = {-1, -1, -1};
  if (g->prof.on) {
    for (int k = 0; k < 3; ++k) {
      evs[k] = prof_event(g);
      mi[k] = (int)g->prof.used - 1;
    }
    ev = evs;
  }
  launch_recon(q, g->prec, g->U[g->cur], flags, z0, z1, g->X, g->Y, g->XY, g->W, g->s, ev);
  prof_span(g, K_RX, m0, mi[0]);
  prof_span(g, K_RY, mi[0], mi[1]);
  if (q.dim == 3) prof_span(g, K_RZ, mi[1], mi[2]);
  int last = q.dim == 3 ? mi[2] : mi[1];
  launch_predict_tab(q, g->prec, g->picard, g->W, g->d_scal + 1, z0, z1, g->ptab, g->L, g->FS, g->s);
  int m2 = prof_mark(g);
  prof_span(g, K_PRED, last, m2);
  if (!do_flux) return;
  launch_flux(q, g->prec, g->FS, z0, z1, g->F, g->s);
  int m3 = prof_mark(g);
  prof_span(g, K_FLUX, m2, m3);
  if (!do_update) return;
  const bool post = g->cfg.fallback == 2;
  launch_update(q, g->prec, g->U[g->cur], g->F, g->d_scal + 1, z0, z1, g->U[1 - g->cur],
                post ? g->d_smax2 : g->d_smax, post ? g->d_err2 : g->d_err, g->s);
  if (post) launch_store_fluxes(q, g->prec, g->F, z0, z1, g->Ffb, g->s);
  int m4 = prof_mark(g);
  prof_span(g, K_UPD, m3, m4);
}

// a posteriori fallback after the whole update, then the CFL max and the
// status of the final state
void fallback_passes(awe_grid* g) {
  int a = prof_mark(g);
  launch_fb_passes(g->q, g->U[g->cur], g->U[1 - g->cur], g->Ffb, g->fbflag, g->d_scal + 1, kFallbackPasses, g->s);
  launch_signal_max(g->q, g->U[1 - g->cur], g->d_smax, g->d_err, g->s);
  int b = prof_mark(g);
  prof_span(g, K_MISC, a, b);
}

void fill_ghosts(awe_grid* g, double* U = nullptr, double c = 0.0) {
  int a = prof_mark(g);
  launch_fill_ghosts(g->q, U ? U : g->U[g->cur], g->d_scal + 0, g->d_scal + 1, c, g->s);
  int b = prof_mark(g);
  prof_span(g, K_GHOST, a, b);
}

const unsigned char* gate_flags_for_step(awe_grid* g, const double* U = nullptr) {
  if (!g->cfg.gate) return nullptr;
  int a = prof_mark(g);
  const unsigned char* f = awe::gate_compute_flags(g->gate, g->q, g->prec, U ? U : g->U[g->cur], g->s);
  int b = prof_mark(g);
  prof_span(g, K_GATE, a, b);
  return f;
}

// the Runge-Kutta stage pipeline of one slab: recon of the stage input,
// face values, fluxes, stage combination
void run_slab_rk(awe_grid* g, const double* in, int z0, int z1, const unsigned char* flags,
                 const RKOut& o1, const RKOut& o2, int nout, bool last) {
  const Geo& q = g->q;
  poison_slab_buffers(g);
  int m0 = prof_mark(g);
  cudaEvent_t evs[3];
  cudaEvent_t* ev = nullptr;
  int mi[3] = {-1, -1, -1};
  if (g->prof.on) {
    for (int k = 0; k < 3; ++k) {
      evs[k] = prof_event(g);
      mi[k] = (int)g->prof.used - 1;
    }
    ev = evs;
  }
  launch_recon(q, g->prec, in, flags, z0, z1, g->X, g->Y, g->XY, g->W, g->s, ev);
  prof_span(g, K_RX, m0, mi[0]);
  prof_span(g, K_RY, mi[0], mi[1]);
  if (q.dim == 3) prof_span(g, K_RZ, mi[1], mi[2]);
  int m1 = q.dim == 3 ? mi[2] : mi[1];
  launch_face_eval(q, g->prec, g->W, z0, z1, g->ptab, g->L, g->FS, g->s);
  int m2 = prof_mark(g);
  prof_span(g, K_FACE, m1, m2);
  launch_rk_flux(q, g->prec, g->FS, z0, z1, g->F, g->s);
  int m3 = prof_mark(g);
  prof_span(g, K_FLUX, m2, m3);
  launch_rk_update(q, g->prec, g->U[g->cur], in, g->F, g->d_scal + 1, z0, z1, o1, o2, nout,
                   last ? g->d_smax : nullptr, g->d_err, g->s);
  int m4 = prof_mark(g);
  prof_span(g, K_UPD, m3, m4);
}

// Stage plan of a Shu-Osher scheme: at stage input k, the outputs are the
// stages i > k with alpha_ik or beta_ik nonzero (k = 0: beta_i0 nonzero, or
// i = 1); a stage's U(0) term alpha_i0 U(0) enters with its first output.
// Buffers: U(0) is the current state, the last stage the other state buffer,
// the others come from the two Runge-Kutta buffers and return there once
// their stage has served as input.  Returns false if a plan needs more than
// two outputs per input or more than two buffers.
struct RKPlan {
  int nout[kRKMax];
  int stage[kRKMax][2];
  int buf[kRKMax + 1];  // -1: U(0); 0, 1: Urk; 2: the output state
};
bool rk_plan(const RKScheme& r, RKPlan& p) {
  bool started[kRKMax + 1] = {false};
  bool used[2] = {false, false};
  p.buf[0] = -1;
  for (int i = 1; i <= r.s; ++i) p.buf[i] = -2;
  for (int k = 0; k < r.s; ++k) {
    p.nout[k] = 0;
    for (int i = k + 1; i <= r.s; ++i) {
      bool contrib = k == 0 ? (i == 1 || r.beta[i][0] != 0.0) : (r.alpha[i][k] != 0.0 || r.beta[i][k] != 0.0);
      if (!contrib) continue;
      if (p.nout[k] == 2) return false;
      if (!started[i]) {
        if (i == r.s) {
          p.buf[i] = 2;
        } else {
          int b = !used[0] ? 0 : !used[1] ? 1 : -1;
          if (b < 0) return false;
          used[b] = true;
          p.buf[i] = b;
        }
        started[i] = true;
      }
      p.stage[k][p.nout[k]++] = i;
    }
    // the stage completed here comes first
    if (p.nout[k] == 0 || p.stage[k][0] != k + 1) {
      if (p.nout[k] == 2 && p.stage[k][1] == k + 1) std::swap(p.stage[k][0], p.stage[k][1]);
      else return false;
    }
    if (k >= 1 && p.buf[k] >= 0 && p.buf[k] < 2) used[p.buf[k]] = false;
  }
  return true;
}

double* rk_buffer(awe_grid* g, int b) { return b == -1 ? g->U[g->cur] : b == 2 ? g->U[1 - g->cur] : g->Urk[b]; }

// Stage k of a Runge-Kutta step: reads the stage input buffer of the plan,
// writes or accumulates into the stages it feeds.  An output stage starts
// (init) at the first input stage that contributes to it.
int rk_stage(awe_grid* g, int k) {
  const RKScheme& r = g->rk;
  RKPlan p;
  if (!rk_plan(r, p)) return fail(g, AWE_ERR_STATE, "Runge-Kutta stage plan");
  bool started[kRKMax + 1] = {false};
  for (int kk = 0; kk < k; ++kk)
    for (int j = 0; j < p.nout[kk]; ++j) started[p.stage[kk][j]] = true;
  double* in = rk_buffer(g, p.buf[k]);
  fill_ghosts(g, in, r.c[k]);
  const unsigned char* flags = gate_flags_for_step(g, in);
  RKOut o[2];
  for (int j = 0; j < p.nout[k]; ++j) {
    int i = p.stage[k][j];
    o[j].out = rk_buffer(g, p.buf[i]);
    o[j].init = started[i] ? 0 : 1;
    o[j].a0 = r.alpha[i][0];
    o[j].al = k == 0 ? 0.0 : r.alpha[i][k];
    o[j].be = r.beta[i][k];
  }
  if (p.nout[k] < 2) o[1] = o[0];
  for (int sidx = 0; sidx < nslabs(g); ++sidx) {
    int z0, z1;
    slab_range(g, sidx, z0, z1);
    run_slab_rk(g, in, z0, z1, flags, o[0], o[1], p.nout[k], k == r.s - 1);
  }
  return AWE_OK;
}

int stage_count(const awe_grid* g) { return g->cfg.scheme == AWE_SCHEME_SSPRK ? g->rk.s : 1; }

// the state buffer that stage k reads, and the time offset (in units of dt) of
// its boundary values
double* stage_input(awe_grid* g, int k, double* c) {
  if (g->cfg.scheme != AWE_SCHEME_SSPRK) {
    *c = 0.0;
    return g->U[g->cur];
  }
  RKPlan p;
  rk_plan(g->rk, p);
  *c = g->rk.c[k];
  return rk_buffer(g, p.buf[k]);
}

bool has_exchange(const awe_grid* g) {
  const int od = g->q.dim - 1;
  return g->q.bc[2 * od] == AWE_BC_EXCHANGE || g->q.bc[2 * od + 1] == AWE_BC_EXCHANGE;
}

// one stage of the current step (the caller checked k == g->next_stage)
int run_stage(awe_grid* g, int k, double dt) {
  if (g->cfg.gate && !g->gate.have_weights) return fail(g, AWE_ERR_STATE, "gate enabled without weights");
  if (k == 0) {
    if (g->poison) {
      const size_t nbytesU = sizeof(double) * g->q.nv * g->q.ntot;
      cudaMemsetAsync(g->U[1 - g->cur], 0xFF, nbytesU, g->s);
      for (int b = 0; b < 2; ++b)
        if (g->Urk[b]) cudaMemsetAsync(g->Urk[b], 0xFF, nbytesU, g->s);
    }
    if (dt > 0) launch_set_scalar(g->d_scal + 1, dt, g->s);
  }
  if (g->cfg.scheme == AWE_SCHEME_SSPRK) {
    int rc = rk_stage(g, k);
    if (rc != AWE_OK) return rc;
  } else {
    fill_ghosts(g);
    const unsigned char* flags = gate_flags_for_step(g);
    for (int sidx = 0; sidx < nslabs(g); ++sidx) {
      int z0, z1;
      slab_range(g, sidx, z0, z1);
      run_slab(g, z0, z1, true, true, flags);
    }
    if (g->cfg.fallback == 2) fallback_passes(g);
  }
  g->next_stage = k + 1;
  if (k == stage_count(g) - 1) {
    launch_finalize(g->q, g->d_scal + 0, g->d_scal + 1, g->d_smax, 1, g->s);
    g->cur = 1 - g->cur;
    g->next_stage = 0;
  }
  CK(g, cudaGetLastError());
  return AWE_OK;
}

}  // namespace

// ============================================================================
extern "C" {

const char* awe_last_error(const awe_grid* g) {
  return g ? g->err.c_str() : g_create_error.c_str();
}

int awe_create(const awe_config* cfg, void* stream, awe_grid** out) {
  if (!cfg || !out) return fail(nullptr, AWE_ERR_ARG, "null argument");
  *out = nullptr;
  const awe_config& c = *cfg;
  if (c.dim != 2 && c.dim != 3) return fail(nullptr, AWE_ERR_ARG, "dim must be 2 or 3");
  if (c.order < 2 || c.order > 4) return fail(nullptr, AWE_ERR_ARG, "order must be 2, 3 or 4");
  if (c.gate && c.order == 2) return fail(nullptr, AWE_ERR_ARG, "the gate needs order 3 or 4 (WENO)");
  if (c.prec != AWE_FP64 && c.prec != AWE_FP32_BULK) return fail(nullptr, AWE_ERR_ARG, "bad prec");
  for (int d = 0; d < c.dim; ++d) {
    if (c.n[d] < c.order) return fail(nullptr, AWE_ERR_ARG, "each dimension needs at least order zones");
    if (!(c.hi[d] > c.lo[d])) return fail(nullptr, AWE_ERR_ARG, "empty domain");
    if (c.dx[d] < 0.0 || c.dx[d] != c.dx[d]) return fail(nullptr, AWE_ERR_ARG, "negative zone size");
  }
  for (int f = 0; f < 2 * c.dim; ++f) {
    if (c.bc[f] < 0 || c.bc[f] > AWE_BC_EXCHANGE) return fail(nullptr, AWE_ERR_ARG, "bad boundary condition");
    if (c.bc[f] == AWE_BC_EXCHANGE && f / 2 != c.dim - 1)
      return fail(nullptr, AWE_ERR_ARG, "AWE_BC_EXCHANGE only on the faces of the outermost dimension");
    // the gate's flag of a ghost zone needs a feature stencil and dilation
    // reaching beyond the g ghost planes: the two subdomains beside an
    // exchanged face would reconstruct its zones with different weights
    if (c.bc[f] == AWE_BC_EXCHANGE && c.gate)
      return fail(nullptr, AWE_ERR_ARG, "the gate cannot be combined with AWE_BC_EXCHANGE");
    // the a posteriori fallback's flags would have to cross exchanged faces
    if (c.bc[f] == AWE_BC_EXCHANGE && c.fallback == 2)
      return fail(nullptr, AWE_ERR_ARG, "fallback 2 cannot be combined with AWE_BC_EXCHANGE");
  }
  if (c.fallback < 0 || c.fallback > 2) return fail(nullptr, AWE_ERR_ARG, "fallback must be 0, 1 or 2");
  if (c.fallback == 2 && c.scheme != AWE_SCHEME_ADER)
    return fail(nullptr, AWE_ERR_ARG, "fallback 2 (a posteriori) is defined for the ADER scheme");
  if (!(c.gamma > 1.0)) return fail(nullptr, AWE_ERR_ARG, "gamma must exceed 1");
  if (c.picard < 0 || c.picard > 8) return fail(nullptr, AWE_ERR_ARG, "picard out of range");
  if (c.slab < 0) return fail(nullptr, AWE_ERR_ARG, "negative slab");
  if (c.riemann < AWE_RS_HLLC || c.riemann > AWE_RS_RUSANOV)
    return fail(nullptr, AWE_ERR_ARG, "riemann must be one of AWE_RS_HLLC, AWE_RS_HLL, AWE_RS_HLLEM, AWE_RS_RUSANOV");
  if (c.scheme != AWE_SCHEME_ADER && c.scheme != AWE_SCHEME_SSPRK)
    return fail(nullptr, AWE_ERR_ARG, "scheme must be AWE_SCHEME_ADER or AWE_SCHEME_SSPRK");
  if (c.scheme == AWE_SCHEME_SSPRK && c.rk_stages != 0 && c.rk_stages != 2 && c.rk_stages != 3 && c.rk_stages != 5)
    return fail(nullptr, AWE_ERR_ARG, "rk_stages must be 0, 2, 3 or 5");
  if (c.dim == 3 && c.n[0] * (long long)c.n[1] * c.n[2] > (1LL << 31))
    return fail(nullptr, AWE_ERR_ARG, "grid too large");
  const char* forced = std::getenv("AWE_FAIL_ALLOC");
  if (forced && forced[0] == '1') return fail(nullptr, AWE_ERR_OOM, "allocation failure forced by AWE_FAIL_ALLOC");

  awe_grid* g = new awe_grid();
  g->cfg = c;
  g->s = (cudaStream_t)stream;
  g->prec = c.prec;
  g->picard = c.picard > 0 ? c.picard : c.order - 1;
  Geo& q = g->q;
  memset(&q, 0, sizeof(q));
  q.dim = c.dim;
  q.N = c.order - 1;
  q.g = c.order;
  q.nv = c.dim + 2;
  for (int d = 0; d < 3; ++d) {
    bool act = d < c.dim;
    q.n[d] = act ? c.n[d] : 1;
    q.G[d] = act ? c.n[d] + 2 * q.g : 1;
    q.dx[d] = act ? (c.dx[d] > 0.0 ? c.dx[d] : (c.hi[d] - c.lo[d]) / c.n[d]) : 1.0;
    q.lo[d] = act ? c.lo[d] : 0.0;
  }
  q.ntot = (long long)q.G[0] * q.G[1] * q.G[2];
  q.gamma = c.gamma;
  q.eps = c.weno_eps;
  q.cfl = c.cfl;
  for (int k = 0; k < 4; ++k) {
    q.lin[k] = c.lin[k];
    q.linf[k] = (float)c.lin[k];
  }
  for (int f = 0; f < 6; ++f) {
    q.bc[f] = f < 2 * c.dim ? c.bc[f] : AWE_BC_PERIODIC;
    for (int v = 0; v < 5; ++v) q.inflow[f][v] = c.inflow[f][v];
  }
  for (int v = 0; v < 5; ++v) q.pre[v] = c.pre[v];
  q.fallback = c.fallback ? 1 : 0;
  q.riemann = c.riemann;
  // the linear-weight reconstruction folded into one stencil per mode: the
  // candidates evaluated on unit differences, combined with the linear weights
  memset(q.lst, 0, sizeof(q.lst));
  memset(q.lstf, 0, sizeof(q.lstf));
  if (q.N >= 2) {
    for (int j = 0; j <= 2 * q.N; ++j) {
      double d[7] = {0, 0, 0, 0, 0, 0, 0};
      d[j] = 1.0;
      double cf[4][3] = {{0}};
      if (q.N == 2) {
        double c2[3][2];
        awe::weno_candidates_n2<double>(d, c2);
        for (int k = 0; k < 3; ++k)
          for (int a = 0; a < 2; ++a) cf[k][a] = c2[k][a];
      } else {
        awe::weno_candidates_n3<double>(d, cf);
      }
      for (int a = 0; a < q.N; ++a) {
        double acc = 0.0;
        for (int k = 0; k <= q.N; ++k) acc += c.lin[k] * cf[k][a];
        q.lst[a][j] = acc;
        q.lstf[a][j] = (float)acc;
      }
    }
  }
  if (c.scheme == AWE_SCHEME_SSPRK) {
    int st = c.rk_stages ? c.rk_stages : (c.order == 2 ? 2 : c.order == 3 ? 3 : 5);
    RKPlan plan;
    if (!rk_scheme(st, g->rk) || !rk_plan(g->rk, plan)) {
      delete g;
      return fail(nullptr, AWE_ERR_ARG, "no Runge-Kutta scheme with that stage count");
    }
  }
  g->slab = (c.dim == 3 && c.slab > 0 && c.slab < c.n[2]) ? c.slab : q.n[2];
  if (c.dim == 2) g->slab = 1;
  g->bytesT = tsize(c.prec);

  auto cleanup_fail = [&](int code) {
    awe_destroy(g);
    return code;
  };
  cudaError_t e = predict_init(g->s);
  if (e != cudaSuccess) {
    int rc = cuda_fail(nullptr, e, "predictor tables");
    delete g;
    return rc;
  }
  Sizes sz = buffer_sizes(q, q.dim == 3 ? g->slab : 1);
  g->szX = sz.X, g->szY = sz.Y, g->szXY = sz.XY, g->szW = sz.W, g->szFS = sz.FS, g->szF = sz.F;
  {
    const char* pz = std::getenv("AWE_POISON");
    g->poison = pz && pz[0] == '1';
  }
  size_t nbytesU = sizeof(double) * q.nv * q.ntot;
  struct A { void** p; size_t n; const char* what; };
  std::vector<A> allocs = {
      {(void**)&g->U[0], nbytesU, "state"},
      {(void**)&g->U[1], nbytesU, "state"},
      {(void**)&g->d_scal, 4 * sizeof(double), "scalars"},
      {(void**)&g->d_smax, sizeof(unsigned long long), "smax"},
      {(void**)&g->d_err, sizeof(int), "err"},
      {(void**)&g->d_fb, sizeof(unsigned long long), "fallback counter"},
      {&g->X, g->bytesT * sz.X, "recon X fields"},
      {&g->Y, g->bytesT * sz.Y, "recon Y fields"},
      {&g->XY, g->bytesT * sz.XY, "recon XY fields"},
      {&g->W, g->bytesT * sz.W, "modes"},
      {&g->FS, g->bytesT * sz.FS, "face states"},
      {&g->F, g->bytesT * sz.F, "fluxes"},
      {(void**)&g->stage, sizeof(double) * q.nv * nactive(q), "staging"},
      {(void**)&g->halo_stage, sizeof(double) * halo_count(q), "halo staging"},
  };
  if (c.scheme == AWE_SCHEME_SSPRK) {
    allocs.push_back({(void**)&g->Urk[0], nbytesU, "Runge-Kutta stage state"});
    allocs.push_back({(void**)&g->Urk[1], nbytesU, "Runge-Kutta stage state"});
  }
  if (c.fallback == 2) {
    long long nff = 0;
    for (int d = 0; d < q.dim; ++d)
      nff += (long long)(q.n[0] + (d == 0)) * (q.n[1] + (d == 1)) * (q.dim == 3 ? q.n[2] + (d == 2) : 1) * q.nv;
    allocs.push_back({(void**)&g->Ffb, sizeof(double) * nff, "whole-grid fluxes (fallback 2)"});
    allocs.push_back({(void**)&g->fbflag, (size_t)nactive(q), "fallback flags"});
    allocs.push_back({(void**)&g->d_smax2, sizeof(unsigned long long), "smax scratch"});
    allocs.push_back({(void**)&g->d_err2, sizeof(int), "status scratch"});
  }
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.n);
    if (e != cudaSuccess) {
      std::string m = std::string("cudaMalloc ") + a.what + " (" + std::to_string(a.n) + " bytes): " + cudaGetErrorString(e);
      g_create_error = m;
      cudaGetLastError();
      return cleanup_fail(AWE_ERR_OOM);
    }
  }
  // node tables of the predictor in the working precision
  g->L = ptab_layout(q.dim, q.N);
  std::vector<double> tab = ptab_build(q.dim, q.N);
  e = cudaMalloc(&g->ptab, g->bytesT * tab.size());
  if (e != cudaSuccess) {
    g_create_error = "cudaMalloc tables";
    return cleanup_fail(AWE_ERR_OOM);
  }
  if (g->prec == AWE_FP64) {
    e = cudaMemcpy(g->ptab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
  } else {
    std::vector<float> tf(tab.begin(), tab.end());
    e = cudaMemcpy(g->ptab, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(g->U[0], 0, nbytesU, g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->U[1], 0, nbytesU, g->s);
  for (int b = 0; b < 2; ++b)
    if (e == cudaSuccess && g->Urk[b]) e = cudaMemsetAsync(g->Urk[b], 0, nbytesU, g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_scal, 0, 4 * sizeof(double), g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_smax, 0, sizeof(unsigned long long), g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_fb, 0, sizeof(unsigned long long), g->s);
  g->q.fb_count = g->d_fb;
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->s);
  if (e != cudaSuccess) {
    g_create_error = std::string("initialisation: ") + cudaGetErrorString(e);
    return cleanup_fail(AWE_ERR_CUDA);
  }
  if (c.gate) {
    int rc = awe::gate_init(g->gate, q, g->s);
    if (rc != AWE_OK) {
      g_create_error = "gate buffers";
      return cleanup_fail(rc);
    }
  }
  *out = g;
  return AWE_OK;
}

int awe_destroy(awe_grid* g) {
  if (!g) return AWE_OK;
  cudaStreamSynchronize(g->s);
  void* ptrs[] = {g->U[0], g->U[1], g->d_scal, g->d_smax,  g->d_err,  g->X,    g->Y,
                  g->XY,   g->W,    g->FS,     g->F,      g->stage,  g->ptab, g->Urk[0],
                  g->Urk[1], g->d_fb, g->halo_stage, g->Ffb, g->fbflag, g->d_smax2, g->d_err2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  awe::gate_free(g->gate);
  for (auto e : g->prof.pool) cudaEventDestroy(e);
  delete g;
  return AWE_OK;
}

// A page-locked host buffer that the device addresses at the same virtual
// address (unified addressing): the scatter / gather kernels then read or
// write it directly over the host link.  That skips the copy engine, whose
// first transfer after an idle period of about a second costs tens of
// milliseconds on this platform.  Anything else (pageable memory) goes through
// the staging buffer with cudaMemcpyAsync.
static bool host_mapped_at(const void* p) {
  // only memory that the CUDA runtime itself page-locked (cudaHostAlloc or
  // cudaHostRegister): on platforms that address pageable memory from the
  // GPU the pointer attributes alone do not tell pinned memory apart
  unsigned int flags = 0;
  if (cudaHostGetFlags(&flags, const_cast<void*>(p)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

// the whole buffer [p, p + bytes): its first and its last element must both be
// page-locked and mapped (a buffer registered over only part of its length,
// such as a view into a larger registration's start, takes the staged copy)
static bool host_mapped(const void* p, size_t bytes) {
  if (!host_mapped_at(p)) return false;
  if (bytes <= sizeof(double)) return true;
  const char* last = static_cast<const char*>(p) + bytes - sizeof(double);
  return host_mapped_at(last);
}

int awe_set_state(awe_grid* g, const double* U, int on_device) {
  if (!g || !U) return fail(g, AWE_ERR_ARG, "null argument");
  const Geo& q = g->q;
  long long n = nactive(q) * q.nv;
  const double* src = U;
  if (!on_device && !host_mapped(U, sizeof(double) * n)) {
    CK(g, cudaMemcpyAsync(g->stage, U, sizeof(double) * n, cudaMemcpyHostToDevice, g->s));
    src = g->stage;
  }
  int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 32);
  k_scatter<<<blocks, 256, 0, g->s>>>(q, src, g->U[g->cur]);
  CK(g, cudaGetLastError());
  if (!on_device) CK(g, cudaStreamSynchronize(g->s));
  return AWE_OK;
}

int awe_get_state(awe_grid* g, double* U, int on_device) {
  if (!g || !U) return fail(g, AWE_ERR_ARG, "null argument");
  const Geo& q = g->q;
  long long n = nactive(q) * q.nv;
  const bool mapped = !on_device && host_mapped(U, sizeof(double) * n);
  double* dst = on_device || mapped ? U : g->stage;
  int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 32);
  k_gather<<<blocks, 256, 0, g->s>>>(q, g->U[g->cur], dst);
  CK(g, cudaGetLastError());
  if (!on_device) {
    if (!mapped) CK(g, cudaMemcpyAsync(U, g->stage, sizeof(double) * n, cudaMemcpyDeviceToHost, g->s));
    CK(g, cudaStreamSynchronize(g->s));
  }
  return AWE_OK;
}

int awe_set_time(awe_grid* g, double t) {
  if (!g) return AWE_ERR_ARG;
  launch_set_scalar(g->d_scal + 0, t, g->s);
  CK(g, cudaGetLastError());
  return AWE_OK;
}

int awe_get_time(awe_grid* g, double* t) {
  if (!g || !t) return fail(g, AWE_ERR_ARG, "null argument");
  CK(g, cudaMemcpyAsync(t, g->d_scal + 0, sizeof(double), cudaMemcpyDeviceToHost, g->s));
  CK(g, cudaStreamSynchronize(g->s));
  return AWE_OK;
}

int awe_cfl_dt(awe_grid* g, double cfl, double* dt_out) {
  if (!g || !(cfl > 0)) return fail(g, AWE_ERR_ARG, "bad argument");
  int a = prof_mark(g);
  launch_signal_max(g->q, g->U[g->cur], g->d_smax, g->d_err, g->s);
  Geo qc = g->q;
  qc.cfl = cfl;
  launch_finalize(qc, g->d_scal + 0, g->d_scal + 1, g->d_smax, 0, g->s);
  int b = prof_mark(g);
  prof_span(g, K_MISC, a, b);
  CK(g, cudaGetLastError());
  if (dt_out) {
    CK(g, cudaMemcpyAsync(dt_out, g->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, g->s));
    CK(g, cudaStreamSynchronize(g->s));
  }
  return AWE_OK;
}

int awe_step(awe_grid* g, double dt, double* dt_next_out) {
  if (!g) return AWE_ERR_ARG;
  if (g->next_stage != 0) return fail(g, AWE_ERR_STATE, "a step is in progress (awe_stage)");
  if (stage_count(g) > 1 && has_exchange(g))
    return fail(g, AWE_ERR_STATE, "exchanged faces need an exchange before every stage: use awe_stage");
  for (int k = 0; k < stage_count(g); ++k) {
    int rc = run_stage(g, k, dt);
    if (rc != AWE_OK) return rc;
  }
  if (dt_next_out) {
    CK(g, cudaMemcpyAsync(dt_next_out, g->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, g->s));
    return awe_check(g);
  }
  return AWE_OK;
}

int awe_stage_count(const awe_grid* g, int* stages) {
  if (!g || !stages) return AWE_ERR_ARG;
  *stages = stage_count(g);
  return AWE_OK;
}

int awe_stage(awe_grid* g, int k, double dt) {
  if (!g) return AWE_ERR_ARG;
  if (k != g->next_stage) return fail(g, AWE_ERR_STATE, "stages run in order: 0, 1, ...");
  return run_stage(g, k, dt);
}

int awe_halo_size(const awe_grid* g, size_t* count) {
  if (!g || !count) return AWE_ERR_ARG;
  *count = (size_t)halo_count(g->q);
  return AWE_OK;
}

int awe_halo_pack(awe_grid* g, int side, double* buf, int on_device) {
  if (!g || !buf || (side != 0 && side != 1)) return fail(g, AWE_ERR_ARG, "bad argument");
  double c = 0.0;
  double* in = stage_input(g, g->next_stage, &c);
  // inner-dimension ghosts of the packed planes, at the stage's boundary time
  fill_ghosts(g, in, c);
  launch_halo(g->q, in, side, on_device ? buf : g->halo_stage, true, g->s);
  CK(g, cudaGetLastError());
  if (!on_device) {
    CK(g, cudaMemcpyAsync(buf, g->halo_stage, sizeof(double) * halo_count(g->q), cudaMemcpyDeviceToHost, g->s));
    CK(g, cudaStreamSynchronize(g->s));
  }
  return AWE_OK;
}

int awe_halo_unpack(awe_grid* g, int side, const double* buf, int on_device) {
  if (!g || !buf || (side != 0 && side != 1)) return fail(g, AWE_ERR_ARG, "bad argument");
  double c = 0.0;
  double* out = stage_input(g, g->next_stage, &c);
  const double* src = buf;
  if (!on_device) {
    CK(g, cudaMemcpyAsync(g->halo_stage, buf, sizeof(double) * halo_count(g->q), cudaMemcpyHostToDevice, g->s));
    src = g->halo_stage;
  }
  launch_halo(g->q, out, side, const_cast<double*>(src), false, g->s);
  CK(g, cudaGetLastError());
  if (!on_device) CK(g, cudaStreamSynchronize(g->s));
  return AWE_OK;
}

int awe_get_dt(awe_grid* g, double* dt, int on_device) {
  if (!g || !dt) return fail(g, AWE_ERR_ARG, "null argument");
  CK(g, cudaMemcpyAsync(dt, g->d_scal + 1, sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        g->s));
  if (!on_device) CK(g, cudaStreamSynchronize(g->s));
  return AWE_OK;
}

int awe_set_dt(awe_grid* g, const double* dt, int on_device) {
  if (!g || !dt) return fail(g, AWE_ERR_ARG, "null argument");
  if (on_device) {
    CK(g, cudaMemcpyAsync(g->d_scal + 1, dt, sizeof(double), cudaMemcpyDeviceToDevice, g->s));
  } else {
    if (!(*dt > 0)) return fail(g, AWE_ERR_ARG, "dt must be positive");
    launch_set_scalar(g->d_scal + 1, *dt, g->s);
    CK(g, cudaGetLastError());
  }
  return AWE_OK;
}

int awe_fallback_count(awe_grid* g, long long* zones) {
  if (!g || !zones) return fail(g, AWE_ERR_ARG, "null argument");
  unsigned long long n = 0;
  CK(g, cudaMemcpyAsync(&n, g->d_fb, sizeof(n), cudaMemcpyDeviceToHost, g->s));
  CK(g, cudaMemsetAsync(g->d_fb, 0, sizeof(n), g->s));
  CK(g, cudaStreamSynchronize(g->s));
  *zones = (long long)n;
  return AWE_OK;
}

int awe_check(awe_grid* g) {
  if (!g) return AWE_ERR_ARG;
  int err = 0;
  CK(g, cudaMemcpyAsync(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->s));
  CK(g, cudaStreamSynchronize(g->s));
  if (err) {
    CK(g, cudaMemsetAsync(g->d_err, 0, sizeof(int), g->s));
    return fail(g, AWE_ERR_NONPHYSICAL, "non-physical or non-finite state after the update");
  }
  return AWE_OK;
}

// ---- probes ------------------------------------------------------------------
static int probe_prepare(awe_grid* g, double dt, bool set_dt) {
  if (nslabs(g) != 1) return fail(g, AWE_ERR_STATE, "probes need a single-slab grid");
  if (set_dt && g->cfg.scheme != AWE_SCHEME_ADER)
    return fail(g, AWE_ERR_STATE, "the face-state and flux probes cover the ADER scheme");
  if (set_dt) {
    CK(g, cudaMemcpyAsync(g->d_scal + 2, g->d_scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, g->s));
    launch_set_scalar(g->d_scal + 1, dt, g->s);
  }
  fill_ghosts(g);
  return AWE_OK;
}
static int probe_copy(awe_grid* g, const void* src, long long n, double* dst) {
  if (g->prec == AWE_FP64) {
    CK(g, cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToHost, g->s));
  } else {
    double* tmp = nullptr;
    CK(g, cudaMallocAsync((void**)&tmp, sizeof(double) * n, g->s));
    k_to_double<float><<<1024, 256, 0, g->s>>>((const float*)src, tmp, n);
    CK(g, cudaMemcpyAsync(dst, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, g->s));
    CK(g, cudaFreeAsync(tmp, g->s));
  }
  CK(g, cudaStreamSynchronize(g->s));
  return AWE_OK;
}

int awe_probe_modes(awe_grid* g, double* W) {
  if (!g || !W) return fail(g, AWE_ERR_ARG, "null argument");
  int rc = probe_prepare(g, 0, false);
  if (rc) return rc;
  const unsigned char* flags = gate_flags_for_step(g);
  int z0, z1;
  slab_range(g, 0, z0, z1);
  launch_recon(g->q, g->prec, g->U[g->cur], flags, z0, z1, g->X, g->Y, g->XY, g->W, g->s, nullptr);
  CK(g, cudaGetLastError());
  return probe_copy(g, g->W, buffer_sizes(g->q, g->q.dim == 3 ? g->slab : 1).W, W);
}

int awe_probe_face_states(awe_grid* g, double dt, double* FS) {
  if (!g || !FS || !(dt > 0)) return fail(g, AWE_ERR_ARG, "bad argument");
  int rc = probe_prepare(g, dt, true);
  if (rc) return rc;
  const unsigned char* flags = gate_flags_for_step(g);
  int z0, z1;
  slab_range(g, 0, z0, z1);
  run_slab(g, z0, z1, false, false, flags);
  CK(g, cudaMemcpyAsync(g->d_scal + 1, g->d_scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, g->s));
  CK(g, cudaGetLastError());
  return probe_copy(g, g->FS, buffer_sizes(g->q, g->q.dim == 3 ? g->slab : 1).FS, FS);
}

int awe_probe_fluxes(awe_grid* g, double dt, double* F) {
  if (!g || !F || !(dt > 0)) return fail(g, AWE_ERR_ARG, "bad argument");
  int rc = probe_prepare(g, dt, true);
  if (rc) return rc;
  const unsigned char* flags = gate_flags_for_step(g);
  int z0, z1;
  slab_range(g, 0, z0, z1);
  run_slab(g, z0, z1, true, false, flags);
  CK(g, cudaMemcpyAsync(g->d_scal + 1, g->d_scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, g->s));
  CK(g, cudaGetLastError());
  return probe_copy(g, g->F, buffer_sizes(g->q, g->q.dim == 3 ? g->slab : 1).F, F);
}

// ---- profiling ---------------------------------------------------------------
int awe_profile(awe_grid* g, int enable) {
  if (!g) return AWE_ERR_ARG;
  prof_collect(g);
  g->prof.on = enable != 0;
  if (enable)
    for (int k = 0; k < K_COUNT; ++k) {
      g->prof.launches[k] = 0;
      g->prof.ms[k] = 0.0;
    }
  return AWE_OK;
}
int awe_profile_count(void) { return K_COUNT; }
int awe_profile_read(awe_grid* g, int kind, const char** name, long* launches, double* total_ms) {
  if (!g || kind < 0 || kind >= K_COUNT) return AWE_ERR_ARG;
  prof_collect(g);
  if (name) *name = kKindNames[kind];
  if (launches) *launches = g->prof.launches[kind];
  if (total_ms) *total_ms = g->prof.ms[kind];
  return AWE_OK;
}

// ---- gate --------------------------------------------------------------------
int awe_gate_set_weights(awe_grid* g, const float* params, size_t n) {
  if (!g || !params) return fail(g, AWE_ERR_ARG, "null argument");
  if (!g->cfg.gate) {
    int rc = awe::gate_init(g->gate, g->q, g->s);
    if (rc != AWE_OK) return fail(g, rc, "gate buffers");
  }
  int rc = awe::gate_set_weights(g->gate, g->q, params, n, g->s);
  if (rc != AWE_OK) return fail(g, rc, "gate weights: wrong parameter count");
  return AWE_OK;
}

int awe_gate_features(awe_grid* g, float* feat, int on_device) {
  if (!g || !feat) return fail(g, AWE_ERR_ARG, "null argument");
  if (!g->gate.ready) {
    int rc = awe::gate_init(g->gate, g->q, g->s);
    if (rc != AWE_OK) return fail(g, rc, "gate buffers");
  }
  fill_ghosts(g);
  return awe::gate_features_out(g->gate, g->q, g->U[g->cur], feat, on_device, g->s);
}

int awe_gate_labels(awe_grid* g, double tau, unsigned char* labels, int on_device) {
  if (!g || !labels) return fail(g, AWE_ERR_ARG, "null argument");
  if (!g->gate.ready) {
    int rc = awe::gate_init(g->gate, g->q, g->s);
    if (rc != AWE_OK) return fail(g, rc, "gate buffers");
  }
  fill_ghosts(g);
  return awe::gate_labels_out(g->gate, g->q, g->U[g->cur], tau, labels, on_device, g->s);
}

int awe_gate_flags(awe_grid* g, unsigned char* flags, int on_device) {
  if (!g || !flags) return fail(g, AWE_ERR_ARG, "null argument");
  if (!g->gate.have_weights) return fail(g, AWE_ERR_STATE, "gate weights not set");
  fill_ghosts(g);
  const unsigned char* f = awe::gate_compute_flags(g->gate, g->q, g->prec, g->U[g->cur], g->s);
  size_t n = (size_t)g->q.ntot;
  CK(g, cudaMemcpyAsync(flags, f, n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->s));
  CK(g, cudaStreamSynchronize(g->s));
  return AWE_OK;
}

int awe_gate_stats(awe_grid* g, long* flagged, long* total) {
  if (!g) return AWE_ERR_ARG;
  return awe::gate_stats(g->gate, g->q, flagged, total, g->s);
}

}  // extern "C"
