// K3: vertex-star patch setup (included by patches.cu inside namespace als,
// after patch_node / vertex_coords / mandel_of).
//
// One CTA per vertex v assembles A_v, the restriction of A_(h,gamma) to the
// d*3^d dofs of the vertex star (Sec. 5.1, Eq. viim), from the 2^d cells of the
// star, and inverts it in FP64.  A_v is symmetric, so only its upper triangle is
// kept (packed by rows in shared memory) and it is inverted by the symmetric
// sweep operator: sweeping pivot k maps M to
//   M_ij - M_ik M_kj / M_kk  (i, j != k),   M_ik / M_kk,   -1 / M_kk  (the pivot),
// which keeps M symmetric; sweeping every pivot in order leaves -A_v^-1.  Each
// pivot is the Schur complement of the leading block (as in Cholesky), hence
// positive for SPD A_v; a non-positive pivot is reported as ALS_ENOTSPD.  This
// is half the flops and half the shared memory of an unsymmetric Gauss-Jordan.
//
// Assembly per cell: one thread per sub-node pair i <= j forms the pair's d x d
// block (the pair (j, i) is its transpose).  With a tensor C the product
// C_q eps(phi_b e_be) is formed once per (point, sub-node, component) and reused
// by every a.  FP64 issue is the limit on this GPU (about 1/70 of the FP32 rate),
// so the kernel minimises FP64 operations rather than idle threads: one division
// per pivot per block, no redundant sums.
#pragma once

__host__ __device__ constexpr int tri_row(int np, int i) { return i * np - (i * (i - 1)) / 2; }

template <int DIM, bool TENSOR>
struct SetupCfg {
  static constexpr int NP = Sz<DIM>::NP, NB = Sz<DIM>::NB, NPR = Sz<DIM>::NPR;
  static constexpr int NM = Sz<DIM>::NM, NC = Sz<DIM>::NC, NSUB = 1 << DIM;
  static constexpr int NPK = NP * (NP + 1) / 2;
  // shared doubles: M | pk | gt | bt | wq | T
  static constexpr int n_M = NPK, n_pk = NP, n_gt = NB * NB * DIM, n_bt = NPR * DIM * NB;
  static constexpr int n_wq = NB * (TENSOR ? NC : 1);
  static constexpr int n_T = TENSOR ? NB * NSUB * DIM * NM : 0;
  static constexpr size_t smem = sizeof(double) * (n_M + n_pk + n_gt + n_bt + n_wq + n_T);
  static constexpr int THREADS = DIM == 3 ? 256 : 128;
};

// patch offset o_k and cell-local index a_k of sub-node bit b_k in a cell on side s_k
//   s_k = 0 (cell below the vertex): o_k = b_k,     a_k = o_k + 1
//   s_k = 1 (cell above):            o_k = b_k + 1, a_k = o_k - 1
template <int DIM>
__device__ __forceinline__ void sub_node(int i, int sx, int sy, int sz, int& P, int& a) {
  const int sv[3] = {sx, sy, sz};
  int o[3], al[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int b = (i >> k) & 1;
    o[k] = sv[k] ? b + 1 : b;
    al[k] = sv[k] ? o[k] - 1 : o[k] + 1;
  }
  P = o[0] + 3 * o[1] + (DIM == 3 ? 9 * o[2] : 0);
  a = al[0] + 3 * al[1] + (DIM == 3 ? 9 * al[2] : 0);
}

// coef: scalar mu [cell][3^d] or Mandel tensor C [cell][3^d][NC] (upper triangle, row-major)
template <int DIM, bool TENSOR>
__global__ void k_patch_setup(Geom g, double gamma, const double* __restrict__ coef, double* __restrict__ inv64,
                              float* __restrict__ inv32, int pstride, DevStatus* st,
                              const double* __restrict__ winv) {
  using C = SetupCfg<DIM, TENSOR>;
  constexpr int NP = C::NP, NB = C::NB, NPR = C::NPR, NM = C::NM, NC = C::NC, NSUB = C::NSUB;
  extern __shared__ double sm[];
  __shared__ double s_dinv;
  double* M = sm;                    // packed upper triangle of the patch matrix, swept in place
  double* pk = M + C::n_M;           // pivot column of the current sweep
  double* gt = pk + C::n_pk;         // [q][a][k] physical gradient of phi_a at point q
  double* bt = gt + C::n_gt;         // [p][alpha][a]: B_K entries, -(psi_p, d phi_a / d x_alpha)_K
  double* wq = bt + C::n_bt;         // [q] |J| w_q mu_q, or [q][NC] |J| w_q C_q, of the current cell
  double* T = wq + C::n_wq;          // tensor: [q][j][be][m] = (C_q eps(phi_b(j) e_be))_m
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const long long v = blockIdx.x;
  int vx, vy, vz;
  vertex_coords<DIM>(g, v, vx, vy, vz);

  double s[3] = {2.0 / g.h[0], 2.0 / g.h[1], DIM == 3 ? 2.0 / g.h[2] : 0.0};
  double wdet = 1.0, vol = 1.0;
  for (int k = 0; k < DIM; ++k) { wdet *= 0.5 * g.h[k]; vol *= g.h[k]; }

  for (int e = tid; e < C::NPK; e += nt) M[e] = 0.0;
  for (int e = tid; e < NB * NB; e += nt) {
    const int q = e / NB, a = e % NB;
    const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    const double bx = Ref<double>::B(qx, ax), by = Ref<double>::B(qy, ay);
    const double bz = DIM == 3 ? Ref<double>::B(qz, az) : 1.0;
    gt[e * DIM + 0] = Ref<double>::D(qx, ax) * by * bz * s[0];
    gt[e * DIM + 1] = bx * Ref<double>::D(qy, ay) * bz * s[1];
    if (DIM == 3) gt[e * DIM + 2] = bx * by * Ref<double>::D(qz, az) * s[2];
  }
  __syncthreads();
  for (int e = tid; e < NPR * DIM * NB; e += nt) {
    const int p = e / (DIM * NB), al = (e / NB) % DIM, a = e % NB;
    double acc = 0.0;
    for (int q = 0; q < NB; ++q) {
      const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
      const double w = wdet * Ref<double>::W(qx) * Ref<double>::W(qy) * (DIM == 3 ? Ref<double>::W(qz) : 1.0);
      const double psi = p == 0 ? 1.0 : Ref<double>::G(p == 1 ? qx : (p == 2 ? qy : qz));
      acc += w * psi * gt[(q * NB + a) * DIM + al];
    }
    bt[e] = -acc;
  }

  // contributions of the 2^d cells of the star
  for (int sc = 0; sc < NSUB; ++sc) {
    const int sx = sc & 1, sy = (sc >> 1) & 1, sz = (sc >> 2) & 1;
    const int cx = vx - 1 + sx, cy = vy - 1 + sy, cz = DIM == 3 ? vz - 1 + sz : 0;
    const bool valid = cx >= 0 && cx < g.n[0] && cy >= 0 && cy < g.n[1] &&
                       (DIM == 2 || (cz >= 0 && cz < g.n[2]));
    __syncthreads();
    if (!valid) continue;
    const long long cell = (long long)cx + (long long)g.n[0] * ((long long)cy + (long long)g.n[1] * cz);
    for (int e = tid; e < C::n_wq; e += nt) {
      const int q = TENSOR ? e / NC : e;
      const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
      wq[e] = wdet * Ref<double>::W(qx) * Ref<double>::W(qy) * (DIM == 3 ? Ref<double>::W(qz) : 1.0) *
              coef[cell * C::n_wq + e];
    }
    __syncthreads();
    if constexpr (TENSOR) {
      // T[q][j][be] = C_q eps(phi_b e_be), b the cell-local node of sub-node j
      for (int e = tid; e < NB * NSUB * DIM; e += nt) {
        const int q = e / (NSUB * DIM), j = (e / DIM) % NSUB, be = e % DIM;
        int Q, b;
        sub_node<DIM>(j, sx, sy, sz, Q, b);
        double eB[NM];
        mandel_of<DIM>(be, gt + (q * NB + b) * DIM, eB);
        const double* Cq = wq + q * NC;
        double* t = T + e * NM;
        for (int m = 0; m < NM; ++m) {
          double acc = 0.0;
          for (int n = 0; n < NM; ++n) {
            const int lo = m < n ? m : n, hi = m < n ? n : m;
            acc += Cq[lo * NM - (lo * (lo - 1)) / 2 + (hi - lo)] * eB[n];
          }
          t[m] = acc;
        }
      }
      __syncthreads();
    }
    // one thread per sub-node pair i <= j: the d x d block of the pair, entries stored at
    // (min(row, col), max(row, col)); the pair (j, i) is the transpose and is skipped
    for (int pr = tid; pr < NSUB * NSUB; pr += nt) {
      const int i = pr / NSUB, j = pr % NSUB;
      if (i > j) continue;
      int P, a, Q, b;
      sub_node<DIM>(i, sx, sy, sz, P, a);
      sub_node<DIM>(j, sx, sy, sz, Q, b);
      long long ndP, ndQ;
      if (!patch_node<DIM>(g, vx, vy, vz, P, ndP) || !patch_node<DIM>(g, vx, vy, vz, Q, ndQ)) continue;
      double V[DIM][DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int l = 0; l < DIM; ++l) V[k][l] = 0.0;
      if constexpr (!TENSOR) {
        // 2 mu eps(phi_b e_be) : eps(phi_a e_al) = mu (d_be phi_a d_al phi_b + delta_(al,be) grad phi_a . grad phi_b)
        double G[DIM][DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k)
#pragma unroll
          for (int l = 0; l < DIM; ++l) G[k][l] = 0.0;
        for (int q = 0; q < NB; ++q) {
          const double w = wq[q];
          const double* ga = gt + (q * NB + a) * DIM;
          const double* gb = gt + (q * NB + b) * DIM;
#pragma unroll
          for (int k = 0; k < DIM; ++k) {
            const double wa = w * ga[k];
#pragma unroll
            for (int l = 0; l < DIM; ++l) G[k][l] += wa * gb[l];
          }
        }
        double tr = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) tr += G[k][k];
#pragma unroll
        for (int al = 0; al < DIM; ++al)
#pragma unroll
          for (int be = 0; be < DIM; ++be) V[al][be] = G[be][al] + (al == be ? tr : 0.0);
      } else {
        for (int q = 0; q < NB; ++q) {
          double eA[DIM][NM];
#pragma unroll
          for (int al = 0; al < DIM; ++al) mandel_of<DIM>(al, gt + (q * NB + a) * DIM, eA[al]);
          const double* t = T + (q * NSUB + j) * DIM * NM;
#pragma unroll
          for (int al = 0; al < DIM; ++al)
#pragma unroll
            for (int be = 0; be < DIM; ++be) {
              double acc = 0.0;
#pragma unroll
              for (int m = 0; m < NM; ++m) acc += eA[al][m] * t[be * NM + m];
              V[al][be] += acc;
            }
        }
      }
#pragma unroll
      for (int al = 0; al < DIM; ++al)
#pragma unroll
        for (int be = 0; be < DIM; ++be) {
          const int row = al * NB + P, col = be * NB + Q;
          if (i == j && row > col) continue;   // the diagonal block: upper triangle only
          double alv = 0.0, val = V[al][be];
          if (winv) {   // gamma B_K^T W_K^-1 B_K with W = M_p(1/mu)
            for (int p = 0; p < NPR; ++p)
              for (int p2 = 0; p2 < NPR; ++p2)
                alv += bt[(p * DIM + al) * NB + a] * winv[(cell * NPR + p) * NPR + p2] * bt[(p2 * DIM + be) * NB + b];
            val += gamma * alv;
          } else {      // W = M_p = |K| diag(1, 1/3, ..)
            for (int p = 0; p < NPR; ++p)
              alv += (p == 0 ? 1.0 : 3.0) * bt[(p * DIM + al) * NB + a] * bt[(p * DIM + be) * NB + b];
            val += gamma / vol * alv;
          }
          const int lo = row < col ? row : col, hi = row < col ? col : row;
          M[tri_row(NP, lo) + (hi - lo)] += val;
        }
    }
  }
  __syncthreads();
  // identity rows for nodes outside the domain or on the Dirichlet boundary
  for (int i = tid; i < NP; i += nt) {
    long long nd;
    if (!patch_node<DIM>(g, vx, vy, vz, i % NB, nd)) M[tri_row(NP, i)] = 1.0;
  }
  __syncthreads();

  // symmetric sweep of every pivot in order: M -> -A_v^-1
  for (int k = 0; k < NP; ++k) {
    for (int i = tid; i < NP; i += nt)
      pk[i] = (i == k) ? 0.0 : M[i < k ? tri_row(NP, i) + (k - i) : tri_row(NP, k) + (i - k)];
    if (tid == 0) {   // one FP64 division per pivot, not one per thread
      double d = M[tri_row(NP, k)];
      if (!(d > 0.0)) {
        report(st, 4 /* ALS_ENOTSPD */, v);
        d = 1.0;
      }
      s_dinv = 1.0 / d;
    }
    __syncthreads();
    const double dinv = s_dinv;
    for (int i = warp; i < NP; i += nwarps) {
      if (i == k) continue;
      const double pi = pk[i] * dinv;
      double* row = M + tri_row(NP, i) - i;
      for (int j = i + lane; j < NP; j += 32)
        if (j != k) row[j] -= pi * pk[j];
    }
    for (int i = tid; i < NP; i += nt) {
      if (i == k) M[tri_row(NP, k)] = -dinv;
      else M[i < k ? tri_row(NP, i) + (k - i) : tri_row(NP, k) + (i - k)] = pk[i] * dinv;
    }
    __syncthreads();
  }
  // A_v^-1 = -M, packed by diagonals in FP64 and block-packed in FP32
  if (inv32) {
    constexpr BlockLayout BLp = BlockLayout(NP);
    for (int e = 44 * BLp.nbp + BLp.nbp + tid; e < BLp.q2; e += nt) inv32[v * pstride + e] = 0.f;
  }
  for (int e = tid; e < C::NPK; e += nt) {
    int t = 0;
    while (diag_start(NP, t + 1) <= e) ++t;
    const int i = e - diag_start(NP, t), j = i + t;
    const double val = -M[tri_row(NP, i) + t];
    if (inv64) inv64[v * pstride + e] = val;
    if (inv32) inv32[v * pstride + BlockLayout(NP).index(i, j)] = (float)val;
  }
}
