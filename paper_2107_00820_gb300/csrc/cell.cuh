// Per-cell sum-factorised evaluation of the augmented Stokes operators.
//
// For one cell K this computes, matrix-free,
//   y_K  = A_K u_K + gamma B_K^T M_K^-1 B_K u_K + B_K^T p_K     (Eqs. (stokessys), (augstokessys))
//   Bu_K = B_K u_K = -(psi, div u)_K
// with [A]_ij = (2 mu eps(phi_i), eps(phi_j)) (scalar mu) or (C eps(phi_j), eps(phi_i))
// (4th-order tensor C, Eq. (stokes-lin)), [B]_ij = -(psi_i, div phi_j) and
// W = M_p block-diagonal over cells.  The AL term stays cell-local: with the
// orthogonal pressure basis {1, xi, eta, zeta}, M_K = |K| diag(1, 1/3, ..) and
// B_K^T M_K^-1 B_K u = (Pi div u, div v)_K, Pi the L2 projection onto P1(K).
// It is fused at the quadrature points: sigma = 2 mu eps(u) + (gamma Pi div u - p) I.
//
// Gradients at the 3^d Gauss points are evaluated by sum factorisation with
// the 1D tables B (values) and D (derivatives), one axis at a time
// (operator.cu).
#pragma once
#include "common.cuh"

namespace als {

enum OpMode : int {
  OP_VISC = 1,   // viscous term (2 mu eps or C eps)
  OP_AL = 2,     // gamma B^T M_p^-1 B
  OP_BT = 4,     // add B^T p
  OP_B = 8,      // write B u
  OP_RAW = 16,   // no Dirichlet constraint (unconstrained operator, used to lift boundary data)
};

// ---------------------------------------------------------------------------
// stress at one point from the velocity gradient g[c][k] = d u_c / d x_k
// ---------------------------------------------------------------------------
template <typename T, int DIM, bool TENSOR>
__device__ __forceinline__ void stress(const T* __restrict__ coef, const T (&g)[DIM][DIM], T iso,
                                       T (&sg)[DIM][DIM]) {
  if constexpr (!TENSOR) {
    const T mu = coef[0];
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int k = 0; k < DIM; ++k) sg[c][k] = mu * (g[c][k] + g[k][c]);
  } else {
    // Mandel vectors: 2D (e00, e11, r2 e01); 3D (e00, e11, e22, r2 e12, r2 e02, r2 e01)
    const T r2 = T(1.4142135623730950488);
    constexpr int NM = Sz<DIM>::NM;
    T e[NM];
    if constexpr (DIM == 2) {
      e[0] = g[0][0]; e[1] = g[1][1]; e[2] = r2 * T(0.5) * (g[0][1] + g[1][0]);
    } else {
      e[0] = g[0][0]; e[1] = g[1][1]; e[2] = g[2][2];
      e[3] = r2 * T(0.5) * (g[1][2] + g[2][1]);
      e[4] = r2 * T(0.5) * (g[0][2] + g[2][0]);
      e[5] = r2 * T(0.5) * (g[0][1] + g[1][0]);
    }
    T sm[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) sm[i] = T(0);
    int idx = 0;
#pragma unroll
    for (int i = 0; i < NM; ++i)
#pragma unroll
      for (int j = i; j < NM; ++j) {
        const T cij = coef[idx++];
        sm[i] += cij * e[j];
        if (j != i) sm[j] += cij * e[i];
      }
    const T ir2 = T(0.70710678118654752440);
    if constexpr (DIM == 2) {
      sg[0][0] = sm[0]; sg[1][1] = sm[1]; sg[0][1] = sg[1][0] = sm[2] * ir2;
    } else {
      sg[0][0] = sm[0]; sg[1][1] = sm[1]; sg[2][2] = sm[2];
      sg[1][2] = sg[2][1] = sm[3] * ir2;
      sg[0][2] = sg[2][0] = sm[4] * ir2;
      sg[0][1] = sg[1][0] = sm[5] * ir2;
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) sg[c][c] += iso;
}

}  // namespace als
