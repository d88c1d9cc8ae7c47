// Newton's method for the viscoplastic rheology of Sec. 5.3.1: the coefficients of the
// linearised problem at a velocity iterate, evaluated at the Gauss points of every
// multigrid level (rediscretisation, Sec. 5.1).
//
// Rheology: mu(eps_II) = mu_ref tau_y / (2 mu_ref eps_II + tau_y) with eps_II =
// sqrt(eps : eps / 2), eps = sym grad u.  Linearisation (the standard Newton method, the
// stress variable T = 2 mu eps of the current iterate): the fourth-order coefficient
// C = 2 mu [I - (eps (x) T)_sym / (2 eps_II max(tau_y, T_II))], in Mandel vectors
// e = M(eps), t = M(T): C = 2 mu [I - s (e t^T + t e^T) / 2], s = 1 / (2 eps_II max(..)).
//
// A coarse level's Gauss point x lies in the fine cell c = floor(x / h_f) (clamped to the
// last cell), at reference coordinates xi = 2 (x / h_f - c) - 1, where the fine Q2 field
// is evaluated.  Coarse-cell midpoints fall on fine-cell faces, where grad u jumps: the
// point location is formed with separately rounded operations in a fixed order,
// x = (K + (1 + xi_q) / 2) h_l, then x / h_f, so that the face is assigned to a cell by the
// arithmetic alone.
#include <math.h>

#include "level.h"

namespace als {

// quadratic Lagrange polynomials on the nodes -1, 0, 1 and their derivatives
__device__ __forceinline__ void q2_basis(double xi, double (&l)[3], double (&dl)[3]) {
  l[0] = 0.5 * xi * (xi - 1.0);
  l[1] = 1.0 - xi * xi;
  l[2] = 0.5 * xi * (xi + 1.0);
  dl[0] = xi - 0.5;
  dl[1] = -2.0 * xi;
  dl[2] = xi + 0.5;
}

template <int DIM>
__global__ void k_newton_coeffs(Geom fg, Geom lg, const double* __restrict__ u, double mu_ref, double tau_y,
                                double* __restrict__ C, double* __restrict__ mu) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NM = DIM == 3 ? 6 : 3, NC = NM * (NM + 1) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= lg.ncells * NQ) return;
  const int q = (int)(t % NQ);
  const long long cell = t / NQ;
  const long long cc[3] = {cell % lg.n[0], (cell / lg.n[0]) % lg.n[1], DIM == 3 ? cell / ((long long)lg.n[0] * lg.n[1]) : 0};
  const int qi[3] = {q % 3, (q / 3) % 3, q / 9};
  const double gq = sqrt(0.6);   // 3-point Gauss-Legendre abscissae -g, 0, g, g^2 = 3/5
  int fc[3] = {0, 0, 0};
  double L[3][3], D[3][3];
  for (int k = 0; k < 3; ++k) {
    L[k][0] = L[k][1] = L[k][2] = 0.0;
    D[k][0] = D[k][1] = D[k][2] = 0.0;
  }
  for (int k = 0; k < DIM; ++k) {
    const double xq = qi[k] == 0 ? -gq : (qi[k] == 1 ? 0.0 : gq);
    const double hl = __ddiv_rn(1.0, (double)lg.n[k]);
    const double hf = __ddiv_rn(1.0, (double)fg.n[k]);
    const double x = __dmul_rn(__dadd_rn((double)cc[k], __dmul_rn(0.5, __dadd_rn(1.0, xq))), hl);
    const double s = __ddiv_rn(x, hf);
    int c = (int)floor(s);
    if (c > fg.n[k] - 1) c = fg.n[k] - 1;
    if (c < 0) c = 0;
    fc[k] = c;
    const double xi = __dsub_rn(__dmul_rn(2.0, __dsub_rn(s, (double)c)), 1.0);
    q2_basis(xi, L[k], D[k]);
    for (int a = 0; a < 3; ++a) D[k][a] *= 2.0 / hf;
  }
  // grad u at the point: G[a][j] = d u_a / d x_j
  double G[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  const int nz = DIM == 3 ? 3 : 1;
  for (int a2 = 0; a2 < nz; ++a2)
    for (int a1 = 0; a1 < 3; ++a1)
      for (int a0 = 0; a0 < 3; ++a0) {
        const long long nd = node_id(fg, 2 * fc[0] + a0, 2 * fc[1] + a1, DIM == 3 ? 2 * fc[2] + a2 : 0);
        double w[3];
        w[0] = D[0][a0] * L[1][a1] * (DIM == 3 ? L[2][a2] : 1.0);
        w[1] = L[0][a0] * D[1][a1] * (DIM == 3 ? L[2][a2] : 1.0);
        w[2] = DIM == 3 ? L[0][a0] * L[1][a1] * D[2][a2] : 0.0;
        for (int a = 0; a < DIM; ++a) {
          const double ua = u[(long long)a * fg.N + nd];
          for (int j = 0; j < DIM; ++j) G[a][j] += ua * w[j];
        }
      }
  // strain (Mandel: diagonal, then sqrt2 x (12, 02, 01) in 3D / (01) in 2D)
  const double r2 = 1.4142135623730951;
  double e[NM];
  if (DIM == 2) {
    e[0] = G[0][0];
    e[1] = G[1][1];
    e[2] = r2 * 0.5 * (G[0][1] + G[1][0]);
  } else {
    e[0] = G[0][0];
    e[1] = G[1][1];
    e[2] = G[2][2];
    e[3] = r2 * 0.5 * (G[1][2] + G[2][1]);
    e[4] = r2 * 0.5 * (G[0][2] + G[2][0]);
    e[5] = r2 * 0.5 * (G[0][1] + G[1][0]);
  }
  double ee = 0.0;
  for (int i = 0; i < NM; ++i) ee += e[i] * e[i];                  // eps : eps
  const double eII = sqrt(0.5 * ee);
  const double m = mu_ref * tau_y / (2.0 * mu_ref * eII + tau_y);
  mu[t] = m;
  if (!C) return;
  // T = 2 mu eps: t = 2 mu e, T_II = 2 mu eps_II
  const double tII = 2.0 * m * eII;
  const double denom = 2.0 * eII * fmax(tau_y, tII);
  const double sc = denom > 0.0 ? 1.0 / denom : 0.0;
  double* out = C + t * NC;
  int k = 0;
  for (int i = 0; i < NM; ++i)
    for (int j = i; j < NM; ++j) {
      const double ti = 2.0 * m * e[i], tj = 2.0 * m * e[j];
      const double sym = 0.5 * (e[i] * tj + ti * e[j]);
      out[k++] = 2.0 * m * ((i == j ? 1.0 : 0.0) - sc * sym);
    }
}

void newton_coeffs(const Geom& fine, const Geom& level, const double* u, double mu_ref, double tau_y, double* C,
                   double* mu, cudaStream_t s) {
  const long long tot = level.ncells * (fine.dim == 3 ? 27 : 9);
  const unsigned blocks = (unsigned)((tot + 127) / 128);
  if (fine.dim == 3) k_newton_coeffs<3><<<blocks, 128, 0, s>>>(fine, level, u, mu_ref, tau_y, C, mu);
  else k_newton_coeffs<2><<<blocks, 128, 0, s>>>(fine, level, u, mu_ref, tau_y, C, mu);
  count_launch(1);
}

}  // namespace als
