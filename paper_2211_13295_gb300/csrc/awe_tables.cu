// awe_tables.cu -- quadrature and basis tables of the predictor and the face
// quadrature, computed on the host from closed forms and uploaded to constant
// memory (per-dimension factors) or to a per-grid device buffer (per-node
// products used by the direct predictor).
//
// Space: Legendre on the zone [-1/2,1/2] with unit leading coefficient,
//   P0 = 1, P1 = x, P2 = x^2 - 1/12, P3 = x^3 - 3x/20, |P_a|^2 = 1, 1/12, 1/180, 1/2800,
//   dP1 = P0, dP2 = 2 P1, dP3 = 3 P2 + P0/10.
// Time: shifted Legendre on [0,1], L0 = 1, L1 = 2t-1, L2 = 6t^2-6t+1,
//   L3 = 20t^3-30t^2+12t-1, |L_e|^2 = 1/(2e+1); I_e(t) = int_0^t L_e.
// Nodes: Gauss-Legendre, 3 points (+-sqrt(3/5)/2, 0; weights 5/18, 8/18) and
//   4 points (+-sqrt(3/7 -+ (2/7) sqrt(6/5))/2; weights (18 +- sqrt(30))/72),
//   face rule 2 points (+-1/(2 sqrt 3), weights 1/2).
#include <cstring>
#include <vector>

#include "awe_internal.cuh"
#include "awe_tables.h"

namespace awe {

double basisP(int a, double x) {
  switch (a) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return x * x - 1.0 / 12.0;
    case 3: return x * x * x - 0.15 * x;
  }
  return 0.0;
}
double basisL(int e, double t) {
  switch (e) {
    case 0: return 1.0;
    case 1: return 2.0 * t - 1.0;
    case 2: return (6.0 * t - 6.0) * t + 1.0;
    case 3: return ((20.0 * t - 30.0) * t + 12.0) * t - 1.0;
  }
  return 0.0;
}
double basisI(int e, double t) {
  switch (e) {
    case 0: return t;
    case 1: return t * t - t;
    case 2: return ((2.0 * t - 3.0) * t + 1.0) * t;
    case 3: return (((5.0 * t - 10.0) * t + 6.0) * t - 1.0) * t;
  }
  return 0.0;
}
static const double kNormP[4] = {1.0, 1.0 / 12.0, 1.0 / 180.0, 1.0 / 2800.0};
static double derivD(int ap, int a) {  // coefficient of P_a in dP_ap/dx
  if (ap == 1 && a == 0) return 1.0;
  if (ap == 2 && a == 1) return 2.0;
  if (ap == 3 && a == 2) return 3.0;
  if (ap == 3 && a == 0) return 0.1;
  return 0.0;
}

void gauss_nodes(int n, double* x, double* w) {
  if (n == 1) {
    x[0] = 0.0;
    w[0] = 1.0;
  } else if (n == 2) {
    double a = 0.5 / std::sqrt(3.0);
    x[0] = -a; x[1] = a;
    w[0] = w[1] = 0.5;
  } else if (n == 3) {
    double a = 0.5 * std::sqrt(0.6);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = w[2] = 5.0 / 18.0; w[1] = 8.0 / 18.0;
  } else if (n == 4) {
    double r = 2.0 / 7.0 * std::sqrt(1.2);
    double a = 0.5 * std::sqrt(3.0 / 7.0 - r), b = 0.5 * std::sqrt(3.0 / 7.0 + r);
    double wa = (18.0 + std::sqrt(30.0)) / 72.0, wb = (18.0 - std::sqrt(30.0)) / 72.0;
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
  }
}

static void make_tabs(int N, Tabs<double>& t) {
  std::memset(&t, 0, sizeof(t));
  const int n = N + 1;
  double x[4], w[4];
  gauss_nodes(n, x, w);
  for (int a = 0; a <= N; ++a)
    for (int i = 0; i < n; ++i) {
      t.PN[a][i] = basisP(a, x[i]);
      t.WPN[a][i] = w[i] * basisP(a, x[i]) / kNormP[a];
    }
  for (int a = 0; a < N; ++a)
    for (int s = 1; s <= N - a; ++s)
      for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int ap = a + 1; ap <= a + s; ++ap) acc += derivD(ap, a) * basisP(ap, x[i]) / kNormP[ap];
        t.QN[a][s][i] = w[i] * acc;
      }
  for (int e = 0; e <= N; ++e)
    for (int i = 0; i < n; ++i) {
      double tau = x[i] + 0.5;
      t.IT[e][i] = basisI(e, tau);
      t.WLT[e][i] = w[i] * basisL(e, tau) * (2.0 * e + 1.0);
    }
  double xf[2], wf[2];
  gauss_nodes(2, xf, wf);
  for (int a = 0; a <= 3; ++a) {
    for (int q = 0; q < 2; ++q) {
      t.PF[a][q] = basisP(a, xf[q]);
      t.ITF[a][q] = basisI(a, xf[q] + 0.5);
    }
    t.PE[a][0] = basisP(a, -0.5);
    t.PE[a][1] = basisP(a, 0.5);
  }
  t.WF[0] = wf[0];
  t.WF[1] = wf[1];
}

template <typename A, typename B> static void cast_tabs(const Tabs<A>& s, Tabs<B>& d) {
  const A* ps = reinterpret_cast<const A*>(&s);
  B* pd = reinterpret_cast<B*>(&d);
  static_assert(sizeof(Tabs<A>) / sizeof(A) == sizeof(Tabs<B>) / sizeof(B), "layout");
  for (size_t i = 0; i < sizeof(Tabs<A>) / sizeof(A); ++i) pd[i] = (B)ps[i];
}

void build_tabs(Tabs<double>* td, Tabs<float>* tf) {
  for (int k = 0; k < 3; ++k) {
    make_tabs(k + 1, td[k]);
    cast_tabs(td[k], tf[k]);
  }
}

// ---------------------------------------------------------------------------
// mode enumerations (same order as the probes document)
// ---------------------------------------------------------------------------
std::vector<std::array<int, 3>> spatial_modes(int D, int N) {
  std::vector<std::array<int, 3>> m;
  int cmax = D == 3 ? N : 0;
  for (int c = 0; c <= cmax; ++c)
    for (int b = 0; b <= N - c; ++b)
      for (int a = 0; a <= N - b - c; ++a) m.push_back({a, b, c});
  return m;
}
// space-time modes of total degree <= M, (a,b,c,e), time outermost
std::vector<std::array<int, 4>> st_modes(int D, int M) {
  std::vector<std::array<int, 4>> m;
  for (int e = 0; e <= M; ++e) {
    int cmax = D == 3 ? M - e : 0;
    for (int c = 0; c <= cmax; ++c)
      for (int b = 0; b <= M - e - c; ++b)
        for (int a = 0; a <= M - e - b - c; ++a) m.push_back({a, b, c, e});
  }
  return m;
}

// ---------------------------------------------------------------------------
// per-configuration node tables (direct predictor and face evaluation)
// ---------------------------------------------------------------------------
PTabLayout ptab_layout(int D, int N) {
  PTabLayout L;
  const int nn = N + 1;
  L.nsn = D == 2 ? nn * nn : nn * nn * nn;
  L.nnodes = L.nsn * nn;
  L.ns = (int)spatial_modes(D, N).size();
  L.ng = (int)st_modes(D, N - 1).size();
  const int nq = (N + 2) / 2;
  L.nfq = D == 2 ? nq * nq : nq * nq * nq;
  size_t off = 0;
  L.ev = off; off += (size_t)L.nnodes * L.ng;
  L.kp = off; off += (size_t)D * L.nnodes * L.ng;
  L.ks = off; off += (size_t)D * L.nsn * L.ng;
  L.ws = off; off += (size_t)L.nsn * L.ns;
  L.fw = off; off += (size_t)D * 2 * L.nfq * L.ns;
  L.fg = off; off += (size_t)D * 2 * L.nfq * L.ng;
  L.total = off;
  return L;
}

std::vector<double> ptab_build(int D, int N) {
  PTabLayout L = ptab_layout(D, N);
  std::vector<double> t(L.total, 0.0);
  const int nn = N + 1;
  const int nq = (N + 2) / 2;
  double x[4], w[4], xf[2], wf[2];
  gauss_nodes(nn, x, w);
  gauss_nodes(nq, xf, wf);
  auto sm = spatial_modes(D, N);
  auto gm = st_modes(D, N - 1);
  auto node_xyz = [&](int s, int* ix) {
    ix[0] = s % nn;
    ix[1] = (s / nn) % nn;
    ix[2] = D == 3 ? s / (nn * nn) : 0;
  };
  for (int s = 0; s < L.nsn; ++s) {
    int ix[3];
    node_xyz(s, ix);
    double pw = w[ix[0]] * w[ix[1]] * (D == 3 ? w[ix[2]] : 1.0);
    for (int m = 0; m < L.ns; ++m) {
      double v = 1.0;
      for (int d = 0; d < D; ++d) v *= basisP(sm[m][d], x[ix[d]]);
      t[L.ws + (size_t)s * L.ns + m] = v;
    }
    for (int it = 0; it < nn; ++it) {
      double tau = x[it] + 0.5;
      int node = s * nn + it;
      for (int b = 0; b < L.ng; ++b) {
        const auto& be = gm[b];
        double ev = basisI(be[3], tau);
        for (int d = 0; d < D; ++d) ev *= basisP(be[d], x[ix[d]]);
        t[L.ev + (size_t)node * L.ng + b] = ev;
        int deg = be[0] + be[1] + be[2] + be[3];
        int slack = N - deg;
        for (int d = 0; d < D; ++d) {
          // w * [sum_a' D[a'][b_d] P_a'(x_d)/|P_a'|^2] * prod_{o!=d} P_{b_o}/|P_{b_o}|^2 * L_e/|L_e|^2
          double f = pw * w[it] * basisL(be[3], tau) * (2.0 * be[3] + 1.0);
          for (int o = 0; o < D; ++o) {
            if (o == d) {
              double acc = 0.0;
              for (int ap = be[d] + 1; ap <= be[d] + slack; ++ap)
                acc += derivD(ap, be[d]) * basisP(ap, x[ix[d]]) / kNormP[ap];
              f *= acc;
            } else {
              f *= basisP(be[o], x[ix[o]]) / kNormP[be[o]];
            }
          }
          t[L.kp + ((size_t)d * L.nnodes + node) * L.ng + b] = f;
          if (be[3] == 0) {
            // time-independent flux: the time factor sums to 1 over the nodes
            double fs = f / (w[it] * basisL(0, tau));
            t[L.ks + ((size_t)d * L.nsn + s) * L.ng + b] = fs;
          }
        }
      }
    }
  }
  // faces: dir d, side (0: -1/2, 1: +1/2), point q = i1 + 2*(i2 + 2*it) (3D), i1 + 2*it (2D)
  for (int d = 0; d < D; ++d) {
    int t1 = -1, t2 = -1;
    for (int e = 0; e < D; ++e)
      if (e != d) {
        if (t1 < 0) t1 = e; else t2 = e;
      }
    for (int side = 0; side < 2; ++side)
      for (int q = 0; q < L.nfq; ++q) {
        int i1 = q % nq, i2 = D == 3 ? (q / nq) % nq : 0, it = D == 3 ? q / (nq * nq) : q / nq;
        double xi[3] = {0, 0, 0};
        xi[d] = side ? 0.5 : -0.5;
        xi[t1] = xf[i1];
        if (t2 >= 0) xi[t2] = xf[i2];
        double tau = xf[it] + 0.5;
        size_t row = ((size_t)d * 2 + side) * L.nfq + q;
        for (int m = 0; m < L.ns; ++m) {
          double v = 1.0;
          for (int e = 0; e < D; ++e) v *= basisP(sm[m][e], xi[e]);
          t[L.fw + row * L.ns + m] = v;
        }
        for (int b = 0; b < L.ng; ++b) {
          double v = basisI(gm[b][3], tau);
          for (int e = 0; e < D; ++e) v *= basisP(gm[b][e], xi[e]);
          t[L.fg + row * L.ng + b] = v;
        }
      }
  }
  return t;
}

}  // namespace awe
