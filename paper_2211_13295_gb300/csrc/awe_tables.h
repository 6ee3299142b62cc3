// awe_tables.h -- host-side table builders (awe_tables.cu)
#pragma once
#include <array>
#include <cstddef>
#include <vector>

namespace awe {

// Offsets (in elements) of the per-configuration node tables of one (D, N):
//  ev[node][g]        phi_g(x_node) I_{g_t}(tau_node)    node = spatial*NN + time
//  kp[d][node][g]     projection kernel of G-mode g for direction d
//  ks[d][snode][g]    same for a time-independent flux (G-modes with g_t = 0)
//  ws[snode][m]       spatial mode m at spatial node
//  fw[d][side][q][m]  spatial mode m at face point q
//  fg[d][side][q][g]  phi_g I_{g_t} at face point q
struct PTabLayout {
  int nsn, nnodes, ns, ng, nfq;
  size_t ev, kp, ks, ws, fw, fg, total;
};

double basisP(int a, double x);
double basisL(int e, double t);
double basisI(int e, double t);
void gauss_nodes(int n, double* x, double* w);
std::vector<std::array<int, 3>> spatial_modes(int D, int N);
std::vector<std::array<int, 4>> st_modes(int D, int M);
PTabLayout ptab_layout(int D, int N);
std::vector<double> ptab_build(int D, int N);

}  // namespace awe
