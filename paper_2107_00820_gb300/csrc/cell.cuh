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
// the 1D tables B (values) and D (derivatives): plane by plane along the last
// axis, row by row along the middle axis, then point by point.
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

template <typename T, int DIM, bool TENSOR>
struct CellArgs {
  const T* mu;     // [cell][3^d] scalar viscosity, or [cell][3^d][NC] Mandel tensor
  T gamma;
  T s[3];          // 2 / h_k
  T wdet;          // |J| = prod h_k / 2
  T inv_m0, inv_m1;  // 1/|K|, 3/|K|
};

template <typename T, int DIM>
__device__ __forceinline__ T psi_at(int p, int qx, int qy, int qz) {
  if (p == 0) return T(1);
  if (p == 1) return Ref<T>::G(qx);
  if (p == 2) return Ref<T>::G(qy);
  return Ref<T>::G(qz);
}

// ---------------------------------------------------------------------------
// divergence moments m_p = (psi_p, div u)_K, p = 0..d
// ---------------------------------------------------------------------------
template <typename T, int DIM>
__device__ __forceinline__ void div_moments(const T (&u)[DIM][Sz<DIM>::NB], const T s[3], T wdet,
                                            T (&m)[Sz<DIM>::NPR]) {
#pragma unroll
  for (int p = 0; p < Sz<DIM>::NPR; ++p) m[p] = T(0);
  if constexpr (DIM == 2) {
#pragma unroll
    for (int qy = 0; qy < 3; ++qy) {
      T a0[3], a1[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        a0[ax] = T(0); a1[ax] = T(0);
#pragma unroll
        for (int ay = 0; ay < 3; ++ay) {
          a0[ax] += Ref<T>::B(qy, ay) * u[0][ax + 3 * ay];
          a1[ax] += Ref<T>::D(qy, ay) * u[1][ax + 3 * ay];
        }
      }
#pragma unroll
      for (int qx = 0; qx < 3; ++qx) {
        T dv = T(0), e = T(0);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          dv += Ref<T>::D(qx, ax) * a0[ax];
          e += Ref<T>::B(qx, ax) * a1[ax];
        }
        dv = dv * s[0] + e * s[1];
        const T w = wdet * Ref<T>::W(qx) * Ref<T>::W(qy) * dv;
        m[0] += w;
        m[1] += w * Ref<T>::G(qx);
        m[2] += w * Ref<T>::G(qy);
      }
    }
  } else {
#pragma unroll
    for (int qz = 0; qz < 3; ++qz) {
      T u0[9], u1[9], u2[9];  // plane values: B_z u_x, B_z u_y, D_z u_z
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        u0[i] = T(0); u1[i] = T(0); u2[i] = T(0);
#pragma unroll
        for (int az = 0; az < 3; ++az) {
          u0[i] += Ref<T>::B(qz, az) * u[0][i + 9 * az];
          u1[i] += Ref<T>::B(qz, az) * u[1][i + 9 * az];
          u2[i] += Ref<T>::D(qz, az) * u[2][i + 9 * az];
        }
      }
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        T a0[3], a1[3], a2[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          a0[ax] = T(0); a1[ax] = T(0); a2[ax] = T(0);
#pragma unroll
          for (int ay = 0; ay < 3; ++ay) {
            a0[ax] += Ref<T>::B(qy, ay) * u0[ax + 3 * ay];
            a1[ax] += Ref<T>::D(qy, ay) * u1[ax + 3 * ay];
            a2[ax] += Ref<T>::B(qy, ay) * u2[ax + 3 * ay];
          }
        }
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            gx += Ref<T>::D(qx, ax) * a0[ax];
            gy += Ref<T>::B(qx, ax) * a1[ax];
            gz += Ref<T>::B(qx, ax) * a2[ax];
          }
          const T dv = gx * s[0] + gy * s[1] + gz * s[2];
          const T w = wdet * Ref<T>::W(qx) * Ref<T>::W(qy) * Ref<T>::W(qz) * dv;
          m[0] += w;
          m[1] += w * Ref<T>::G(qx);
          m[2] += w * Ref<T>::G(qy);
          m[3] += w * Ref<T>::G(qz);
        }
      }
    }
  }
}

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

// ---------------------------------------------------------------------------
// y_K = sum_q wdet_q sigma(q) : grad phi(q)   with sigma from the modes requested
//   pi[p]  : coefficients of gamma Pi div u - p_K on the basis psi (isotropic part)
// ---------------------------------------------------------------------------
template <typename T, int DIM, bool TENSOR, bool VISC>
__device__ __forceinline__ void cell_flux_apply(const T (&u)[DIM][Sz<DIM>::NB], const T* __restrict__ coef,
                                                const T s[3], T wdet, const T (&pi)[Sz<DIM>::NPR],
                                                T (&y)[DIM][Sz<DIM>::NB]) {
  constexpr int NB = Sz<DIM>::NB;
  constexpr int NCQ = TENSOR ? Sz<DIM>::NC : 1;
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int a = 0; a < NB; ++a) y[c][a] = T(0);

  if constexpr (DIM == 2) {
#pragma unroll
    for (int qy = 0; qy < 3; ++qy) {
      // forward: a0 = B_y u (for d/dx), a1 = D_y u (for d/dy)
      T a0[2][3], a1[2][3];
      if constexpr (VISC) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            a0[c][ax] = T(0); a1[c][ax] = T(0);
#pragma unroll
            for (int ay = 0; ay < 3; ++ay) {
              a0[c][ax] += Ref<T>::B(qy, ay) * u[c][ax + 3 * ay];
              a1[c][ax] += Ref<T>::D(qy, ay) * u[c][ax + 3 * ay];
            }
          }
      }
      T r0[2][3], r1[2][3];  // row accumulators (pair with B_y and D_y)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) { r0[c][ax] = T(0); r1[c][ax] = T(0); }
#pragma unroll
      for (int qx = 0; qx < 3; ++qx) {
        const int q = qx + 3 * qy;
        const T iso = pi[0] + pi[1] * Ref<T>::G(qx) + pi[2] * Ref<T>::G(qy);
        T sg[2][2];
        if constexpr (VISC) {
          T g[2][2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            T gx = T(0), gy = T(0);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              gx += Ref<T>::D(qx, ax) * a0[c][ax];
              gy += Ref<T>::B(qx, ax) * a1[c][ax];
            }
            g[c][0] = gx * s[0]; g[c][1] = gy * s[1];
          }
          stress<T, 2, TENSOR>(coef + q * NCQ, g, iso, sg);
        } else {
          sg[0][0] = iso; sg[1][1] = iso; sg[0][1] = T(0); sg[1][0] = T(0);
        }
        const T w = wdet * Ref<T>::W(qx) * Ref<T>::W(qy);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T f0 = w * sg[c][0] * s[0], f1 = w * sg[c][1] * s[1];
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) {
            r0[c][ax] += Ref<T>::D(qx, ax) * f0;
            r1[c][ax] += Ref<T>::B(qx, ax) * f1;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int ay = 0; ay < 3; ++ay)
#pragma unroll
          for (int ax = 0; ax < 3; ++ax)
            y[c][ax + 3 * ay] += Ref<T>::B(qy, ay) * r0[c][ax] + Ref<T>::D(qy, ay) * r1[c][ax];
    }
  } else {
#pragma unroll 1
    for (int qz = 0; qz < 3; ++qz) {
      T U0[3][9], U1[3][9];   // B_z u, D_z u on the plane
      if constexpr (VISC) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            U0[c][i] = T(0); U1[c][i] = T(0);
#pragma unroll
            for (int az = 0; az < 3; ++az) {
              U0[c][i] += Ref<T>::B(qz, az) * u[c][i + 9 * az];
              U1[c][i] += Ref<T>::D(qz, az) * u[c][i + 9 * az];
            }
          }
      }
      T V0[3][9], V1[3][9];   // plane accumulators (pair with B_z and D_z)
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int i = 0; i < 9; ++i) { V0[c][i] = T(0); V1[c][i] = T(0); }
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        T A0[3][3], A1[3][3], A2[3][3];  // B_y U0 (d/dx), D_y U0 (d/dy), B_y U1 (d/dz)
        if constexpr (VISC) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              A0[c][ax] = T(0); A1[c][ax] = T(0); A2[c][ax] = T(0);
#pragma unroll
              for (int ay = 0; ay < 3; ++ay) {
                A0[c][ax] += Ref<T>::B(qy, ay) * U0[c][ax + 3 * ay];
                A1[c][ax] += Ref<T>::D(qy, ay) * U0[c][ax + 3 * ay];
                A2[c][ax] += Ref<T>::B(qy, ay) * U1[c][ax + 3 * ay];
              }
            }
        }
        T R0[3][3], R1[3][3], R2[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int ax = 0; ax < 3; ++ax) { R0[c][ax] = T(0); R1[c][ax] = T(0); R2[c][ax] = T(0); }
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          const int q = qx + 3 * qy + 9 * qz;
          const T iso = pi[0] + pi[1] * Ref<T>::G(qx) + pi[2] * Ref<T>::G(qy) + pi[3] * Ref<T>::G(qz);
          T sg[3][3];
          if constexpr (VISC) {
            T g[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
              for (int ax = 0; ax < 3; ++ax) {
                gx += Ref<T>::D(qx, ax) * A0[c][ax];
                gy += Ref<T>::B(qx, ax) * A1[c][ax];
                gz += Ref<T>::B(qx, ax) * A2[c][ax];
              }
              g[c][0] = gx * s[0]; g[c][1] = gy * s[1]; g[c][2] = gz * s[2];
            }
            stress<T, 3, TENSOR>(coef + q * NCQ, g, iso, sg);
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int k = 0; k < 3; ++k) sg[c][k] = (c == k) ? iso : T(0);
          }
          const T w = wdet * Ref<T>::W(qx) * Ref<T>::W(qy) * Ref<T>::W(qz);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const T f0 = w * sg[c][0] * s[0], f1 = w * sg[c][1] * s[1], f2 = w * sg[c][2] * s[2];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              R0[c][ax] += Ref<T>::D(qx, ax) * f0;
              R1[c][ax] += Ref<T>::B(qx, ax) * f1;
              R2[c][ax] += Ref<T>::B(qx, ax) * f2;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int ay = 0; ay < 3; ++ay)
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
              V0[c][ax + 3 * ay] += Ref<T>::B(qy, ay) * R0[c][ax] + Ref<T>::D(qy, ay) * R1[c][ax];
              V1[c][ax + 3 * ay] += Ref<T>::B(qy, ay) * R2[c][ax];
            }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int az = 0; az < 3; ++az)
#pragma unroll
          for (int i = 0; i < 9; ++i)
            y[c][i + 9 * az] += Ref<T>::B(qz, az) * V0[c][i] + Ref<T>::D(qz, az) * V1[c][i];
    }
  }
}

}  // namespace als
