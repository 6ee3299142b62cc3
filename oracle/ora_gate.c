/*
 * ora_gate.c -- oracle of the learned troubled-zone gate (TEST INFRASTRUCTURE
 * ONLY; see ora.h).  The paper has no learned part: this follows the gate's
 * definition stated below.  Labels come from the method itself (deviation of
 * the WENO nonlinear weights from the linear weights); the network is a
 * 2x32 ReLU MLP on stencil features; its decision is taken in FP32 with a fixed
 * summation order so that the CUDA path and this oracle reach identical flags.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ora.h"

#define MAXN 3

typedef struct {
  int dim, N, nv;
  int n[3], G[3];
  size_t ntot;
} ggeom;

static void mk(const ora_cfg* c, ggeom* q) {
  q->dim = c->dim;
  q->N = c->order - 1;
  q->nv = c->dim + 2;
  for (int d = 0; d < 3; ++d) {
    q->n[d] = d < c->dim ? c->n[d] : 1;
    q->G[d] = d < c->dim ? c->n[d] + 2 * c->order : 1;
  }
  q->ntot = (size_t)q->G[0] * q->G[1] * q->G[2];
}
static size_t gi(const ggeom* q, int i, int j, int k) { return ((size_t)k * q->G[1] + j) * q->G[0] + i; }
static int stencil_fits(const ggeom* q, const int* idx) {
  for (int d = 0; d < q->dim; ++d)
    if (idx[d] < q->N || idx[d] > q->G[d] - 1 - q->N) return 0;
  return 1;
}

int ora_gate_num_features(int dim, int order) { return dim * 2 * (2 * (order - 1) + 1); }

/* Label of a zone: 1 when, for some direction, for density or total energy,
 * some candidate's nonlinear weight differs from its linear weight by more
 * than tau (the WENO weights of the pure-direction recon of the zone means). */
int ora_weno_labels(const ora_cfg* c, const double* Ug, double tau, unsigned char* labels) {
  ggeom q;
  mk(c, &q);
  const int N = q.N;
  for (int k = 0; k < q.G[2]; ++k)
    for (int j = 0; j < q.G[1]; ++j)
      for (int i = 0; i < q.G[0]; ++i) {
        int idx[3] = {i, j, k};
        size_t z = gi(&q, i, j, k);
        if (!stencil_fits(&q, idx)) { labels[z] = 255; continue; }
        int lab = 0;
        for (int d = 0; d < q.dim; ++d)
          for (int vv = 0; vv < 2; ++vv) {
            int v = vv ? q.nv - 1 : 0;
            double u[2 * MAXN + 1], coef[MAXN], om[MAXN + 1];
            for (int s = -N; s <= N; ++s) {
              int m[3] = {i, j, k};
              m[d] += s;
              u[N + s] = Ug[(size_t)v * q.ntot + gi(&q, m[0], m[1], m[2])];
            }
            ora_weno1d(N, u, c->eps, c->lin, 0, coef, om);
            for (int kk = 0; kk <= N; ++kk)
              if (fabs(om[kk] - c->lin[kk]) > tau) lab = 1;
          }
        labels[z] = (unsigned char)lab;
      }
  return 0;
}

/* Features: for each direction d and for rho and E (the quantities the
 * labels look at), the 2N undivided differences delta_k = f(i+k+1-N) -
 * f(i+k-N), k = 0..2N-1 (FP64), divided by their largest magnitude s (the
 * shape of the stencil, which is what ratios of smoothness indicators see; 0
 * when the data is constant), then one magnitude feature: s over |f(i)| +
 * 1e-12, scaled by 100 and squashed by x/(1+x).  The differences and s are
 * taken in FP64; the divisions, the scaling and the squashing in FP32 on the
 * FP32-rounded values, each operation rounded once (a classifier input needs
 * no more, and both implementations reach the same bits).  Index
 * (d*2 + q)*(2N+1) + k, with k = 2N the magnitude. */
int ora_gate_features(const ora_cfg* c, const double* Ug, float* feat) {
  ggeom q;
  mk(c, &q);
  const int N = q.N, nf = ora_gate_num_features(q.dim, c->order);
  for (int k = 0; k < q.G[2]; ++k)
    for (int j = 0; j < q.G[1]; ++j)
      for (int i = 0; i < q.G[0]; ++i) {
        int idx[3] = {i, j, k};
        size_t z = gi(&q, i, j, k);
        float* f = feat + z * nf;
        if (!stencil_fits(&q, idx)) {
          for (int t = 0; t < nf; ++t) f[t] = 0.0f;
          continue;
        }
        for (int d = 0; d < q.dim; ++d)
          for (int qty = 0; qty < 2; ++qty) {
            int v = qty == 0 ? 0 : q.nv - 1;
            double vals[2 * MAXN + 1], del[2 * MAXN];
            for (int s = -N; s <= N; ++s) {
              int m[3] = {i, j, k};
              m[d] += s;
              vals[N + s] = Ug[(size_t)v * q.ntot + gi(&q, m[0], m[1], m[2])];
            }
            double sc = 0.0;
            for (int t = 0; t < 2 * N; ++t) {
              del[t] = vals[t + 1] - vals[t];
              sc = fmax(sc, fabs(del[t]));
            }
            float* o = f + (d * 2 + qty) * (2 * N + 1);
            const float scf = (float)sc;
            for (int t = 0; t < 2 * N; ++t) o[t] = scf > 0.0f ? (float)del[t] / scf : 0.0f;
            const float den = (float)fabs(vals[N]) + 1e-12f;
            const float x = 100.0f * (scf / den);
            o[2 * N] = x / (1.0f + x);
          }
      }
  return 0;
}

/* Packed parameters: W1[nh][nin], b1[nh], W2[nh][nh], b2[nh], w3[nh], b3. */
size_t ora_mlp_num_params(int nin, int nh) {
  return (size_t)nh * nin + nh + (size_t)nh * nh + nh + nh + 1;
}

void ora_mlp_forward_f64(int nin, int nh, const float* P, const float* x, int B, double* z) {
  const float *W1 = P, *b1 = W1 + (size_t)nh * nin, *W2 = b1 + nh, *b2 = W2 + (size_t)nh * nh,
              *w3 = b2 + nh, *b3 = w3 + nh;
  double h1[64], h2[64];
  for (int b = 0; b < B; ++b) {
    const float* xb = x + (size_t)b * nin;
    for (int j = 0; j < nh; ++j) {
      double a = b1[j];
      for (int i = 0; i < nin; ++i) a += (double)W1[j * nin + i] * xb[i];
      h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int k = 0; k < nh; ++k) {
      double a = b2[k];
      for (int j = 0; j < nh; ++j) a += (double)W2[k * nh + j] * h1[j];
      h2[k] = a > 0.0 ? a : 0.0;
    }
    double o = b3[0];
    for (int k = 0; k < nh; ++k) o += (double)w3[k] * h2[k];
    z[b] = o;
  }
}

/* mean over the batch of the logistic loss log(1+exp(z)) - y z, and its
 * gradient by the chain rule through the two ReLU layers */
double ora_mlp_loss_grad_f64(int nin, int nh, const float* P, const float* x, const float* y, int B,
                             double* grad) {
  const float *W1 = P, *b1 = W1 + (size_t)nh * nin, *W2 = b1 + nh, *b2 = W2 + (size_t)nh * nh,
              *w3 = b2 + nh, *b3 = w3 + nh;
  size_t np = ora_mlp_num_params(nin, nh);
  double *gW1 = grad, *gb1 = gW1 + (size_t)nh * nin, *gW2 = gb1 + nh, *gb2 = gW2 + (size_t)nh * nh,
         *gw3 = gb2 + nh, *gb3 = gw3 + nh;
  memset(grad, 0, np * sizeof(double));
  double loss = 0.0;
  double a1[64], h1[64], a2[64], h2[64], d2[64], d1[64];
  for (int b = 0; b < B; ++b) {
    const float* xb = x + (size_t)b * nin;
    for (int j = 0; j < nh; ++j) {
      double a = b1[j];
      for (int i = 0; i < nin; ++i) a += (double)W1[j * nin + i] * xb[i];
      a1[j] = a;
      h1[j] = a > 0.0 ? a : 0.0;
    }
    for (int k = 0; k < nh; ++k) {
      double a = b2[k];
      for (int j = 0; j < nh; ++j) a += (double)W2[k * nh + j] * h1[j];
      a2[k] = a;
      h2[k] = a > 0.0 ? a : 0.0;
    }
    double zz = b3[0];
    for (int k = 0; k < nh; ++k) zz += (double)w3[k] * h2[k];
    double yy = y[b];
    loss += (zz > 0.0 ? zz : 0.0) - yy * zz + log1p(exp(-fabs(zz)));
    double dz = (1.0 / (1.0 + exp(-zz)) - yy) / B;
    gb3[0] += dz;
    for (int k = 0; k < nh; ++k) {
      gw3[k] += dz * h2[k];
      d2[k] = a2[k] > 0.0 ? dz * w3[k] : 0.0;
      gb2[k] += d2[k];
    }
    for (int j = 0; j < nh; ++j) {
      double s = 0.0;
      for (int k = 0; k < nh; ++k) {
        gW2[k * nh + j] += d2[k] * h1[j];
        s += d2[k] * W2[k * nh + j];
      }
      d1[j] = a1[j] > 0.0 ? s : 0.0;
      gb1[j] += d1[j];
      for (int i = 0; i < nin; ++i) gW1[j * nin + i] += d1[j] * xb[i];
    }
  }
  return loss / B;
}

/* FP32 forward, accumulator started at the bias, inputs taken in index order
 * with a fused multiply-add each (the order the decision is defined in). */
void ora_mlp_forward_f32(int nin, int nh, const float* P, const float* x, int B, float* z) {
  const float *W1 = P, *b1 = W1 + (size_t)nh * nin, *W2 = b1 + nh, *b2 = W2 + (size_t)nh * nh,
              *w3 = b2 + nh, *b3 = w3 + nh;
  float h1[64], h2[64];
  for (int b = 0; b < B; ++b) {
    const float* xb = x + (size_t)b * nin;
    for (int j = 0; j < nh; ++j) {
      float a = b1[j];
      for (int i = 0; i < nin; ++i) a = fmaf(W1[j * nin + i], xb[i], a);
      h1[j] = a > 0.0f ? a : 0.0f;
    }
    for (int k = 0; k < nh; ++k) {
      float a = b2[k];
      for (int j = 0; j < nh; ++j) a = fmaf(W2[k * nh + j], h1[j], a);
      h2[k] = a > 0.0f ? a : 0.0f;
    }
    float o = b3[0];
    for (int k = 0; k < nh; ++k) o = fmaf(w3[k], h2[k], o);
    z[b] = o;
  }
}

/* Gate flags: a zone is troubled when its logit is > 0 (probability > 1/2);
 * zones without a full stencil count as troubled; a zone is sent through full
 * WENO when it or one of its face neighbours is troubled. */
int ora_gate_flags(const ora_cfg* c, const double* Ug, int nh, const float* params, unsigned char* flags) {
  ggeom q;
  mk(c, &q);
  const int nf = ora_gate_num_features(q.dim, c->order);
  float* feat = (float*)malloc(sizeof(float) * nf * q.ntot);
  unsigned char* raw = (unsigned char*)malloc(q.ntot);
  ora_gate_features(c, Ug, feat);
  for (int k = 0; k < q.G[2]; ++k)
    for (int j = 0; j < q.G[1]; ++j)
      for (int i = 0; i < q.G[0]; ++i) {
        int idx[3] = {i, j, k};
        size_t z = gi(&q, i, j, k);
        if (!stencil_fits(&q, idx)) { raw[z] = 1; continue; }
        float lz;
        ora_mlp_forward_f32(nf, nh, params, feat + z * nf, 1, &lz);
        raw[z] = lz > 0.0f ? 1 : 0;
      }
  for (int k = 0; k < q.G[2]; ++k)
    for (int j = 0; j < q.G[1]; ++j)
      for (int i = 0; i < q.G[0]; ++i) {
        size_t z = gi(&q, i, j, k);
        unsigned char f = raw[z];
        for (int d = 0; d < q.dim; ++d)
          for (int s = -1; s <= 1; s += 2) {
            int m[3] = {i, j, k};
            m[d] += s;
            if (m[d] < 0 || m[d] >= q.G[d]) continue;
            f |= raw[gi(&q, m[0], m[1], m[2])];
          }
        flags[z] = f;
      }
  free(feat);
  free(raw);
  return 0;
}
