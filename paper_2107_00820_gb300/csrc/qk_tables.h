// Host-side 1D tables of the order-3 velocity space (Sec. 5.2.2, Table k), shared by the
// 2D and 3D kernels: the cubic Lagrange basis on the equispaced nodes -1, -1/3, 1/3, 1,
// its values and derivatives at the 4-point Gauss-Legendre abscissae, the weights, and
// the prolongation weights (the coarse basis at the fine nodes of a coarse cell).
#pragma once
#include <math.h>

namespace als {
namespace qk_tab {

constexpr int K = 3;        // polynomial order
constexpr int N1 = K + 1;   // nodes (and Gauss points) per axis and cell
constexpr int NF = 2 * K + 1;   // fine lattice nodes per coarse cell and axis

// G[q]: abscissae; L[q][a] = l_a(G[q]), D[q][a] = l_a'(G[q]); W[q]: weights;
// PW[f][a] = l_a(f / K - 1), f = 0..2K (the fine nodes of a coarse cell per axis)
inline void tables_1d(double G[N1], double L[N1][N1], double D[N1][N1], double W[N1], double PW[NF][N1]) {
  // 4-point Gauss-Legendre rule: +-sqrt(3/7 -+ 2/7 sqrt(6/5)), weights (18 +- sqrt(30)) / 36
  const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
  const double g[N1] = {-b, -a, a, b};
  const double w[N1] = {wb, wa, wa, wb};
  const double t[N1] = {-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0};   // Lagrange nodes
  auto lag = [&](int i, double x) {
    double v = 1.0;
    for (int j = 0; j < N1; ++j)
      if (j != i) v *= (x - t[j]) / (t[i] - t[j]);
    return v;
  };
  auto dlag = [&](int i, double x) {
    double s = 0.0;
    for (int m = 0; m < N1; ++m) {
      if (m == i) continue;
      double v = 1.0 / (t[i] - t[m]);
      for (int j = 0; j < N1; ++j)
        if (j != i && j != m) v *= (x - t[j]) / (t[i] - t[j]);
      s += v;
    }
    return s;
  };
  for (int q = 0; q < N1; ++q) {
    G[q] = g[q];
    W[q] = w[q];
    for (int i = 0; i < N1; ++i) {
      L[q][i] = lag(i, g[q]);
      D[q][i] = dlag(i, g[q]);
    }
  }
  for (int f = 0; f < NF; ++f)
    for (int i = 0; i < N1; ++i) PW[f][i] = lag(i, (double)f / K - 1.0);
}

}  // namespace qk_tab
}  // namespace als
