// K3: vertex-star patch setup (included by patches.cu inside namespace als,
// after patch_node / vertex_coords / mandel_of and df64.cuh).
//
// One CTA per vertex v assembles A_v, the restriction of A_(h,gamma) to the
// d*3^d dofs of the vertex star (Sec. 4.1, Eq. viim), from the 2^d cells of the
// star, and inverts it in the arithmetic R: FP64, or double-float (DF64, about 48
// significant bits in FP32 pairs, see df64.cuh) when only the FP32 cycle needs the
// inverse to FP32 accuracy.  A_v is symmetric, so only its upper triangle is
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
  // shared doubles: M | pk | qk | gt | bt | wq | wpsi | T, then the row index of every packed entry
  static constexpr int n_M = NPK, n_pk = NP, n_qk = NP, n_gt = NB * NB * DIM, n_bt = NPR * DIM * NB;
  static constexpr int n_wq = NB * (TENSOR ? NC : 1), n_wpsi = NPR * NB;
  static constexpr int n_T = TENSOR ? NB * NSUB * DIM * NM : 0;
  static constexpr int n_dbl = n_M + n_pk + n_qk + n_gt + n_bt + n_wq + n_wpsi + n_T;
  static constexpr size_t smem = sizeof(double) * n_dbl + NPK;   // + uint8 row index per entry
  static_assert(NP <= 255, "row index stored in 8 bits");
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

// Nonzero Mandel entries of eps(phi e_al) for the gradient gr of phi: slot al with
// d_al phi, and the shear slots of the pairs (al, o) with ir2 = sqrt(1/2) times d_o phi
// (the same entries as mandel_of without its zeros; 3 in 3D, 2 in 2D).  3D shear slots:
// 3 = (1,2), 4 = (0,2), 5 = (0,1); 2D: 2 = (0,1).
template <int DIM, typename R>
__device__ __forceinline__ void strain_nonzeros(int al, const R* gr, R ir2, int (&n)[3], R (&e)[3]) {
  n[0] = al;
  e[0] = gr[al];
  if (DIM == 2) {
    n[1] = 2; e[1] = gr[1 - al] * ir2;
    n[2] = 0; e[2] = gr[al] * R{};   // unused slot
  } else {
    const int o1 = al == 0 ? 1 : 0, o2 = al == 2 ? 1 : 2;      // the two other axes
    n[1] = (al + o1 == 1) ? 5 : ((al + o1 == 2) ? 4 : 3);
    n[2] = (al + o2 == 1) ? 5 : ((al + o2 == 2) ? 4 : 3);
    e[1] = gr[o1] * ir2;
    e[2] = gr[o2] * ir2;
  }
}

// coef: scalar mu [cell][3^d] or Mandel tensor C [cell][3^d][NC] (upper triangle, row-major)
// Level constants computed once on the host: 2/h per axis, |J| = prod h/2, |K|, gamma/|K|
struct SetupGeo {
  double s[3];
  double wdet, vol, gvol;
};

// The level's reference tables, in FP64 and stored in R (one CTA, once per setup):
// wpsi [p][q] = |J| w_q psi_p(q); gt [q][a][k] = d phi_a / d x_k at point q;
// bt [p][alpha][a] = -(psi_p, d phi_a / d x_alpha)_K.  Layout: gt | wpsi | bt.
template <int DIM>
struct SetupTab {
  static constexpr int NB = Sz<DIM>::NB, NPR = Sz<DIM>::NPR;
  static constexpr int n_gt = NB * NB * DIM, n_wpsi = NPR * NB, n_bt = NPR * DIM * NB;
  static constexpr int total = n_gt + n_wpsi + n_bt;
};

template <int DIM, typename R>
__global__ void k_setup_tables(SetupGeo sg, R* __restrict__ tab) {
  using TB = SetupTab<DIM>;
  constexpr int NB = TB::NB, NPR = TB::NPR;
  __shared__ double gt[TB::n_gt], wpsi[TB::n_wpsi];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < NPR * NB; e += nt) {
    const int p = e / NB, q = e % NB;
    const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    const double w = sg.wdet * Ref<double>::W(qx) * Ref<double>::W(qy) * (DIM == 3 ? Ref<double>::W(qz) : 1.0);
    wpsi[e] = p == 0 ? w : w * Ref<double>::G(p == 1 ? qx : (p == 2 ? qy : qz));
  }
  for (int e = tid; e < NB * NB; e += nt) {
    const int q = e / NB, a = e % NB;
    const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
    const double bx = Ref<double>::B(qx, ax), by = Ref<double>::B(qy, ay);
    const double bz = DIM == 3 ? Ref<double>::B(qz, az) : 1.0;
    gt[e * DIM + 0] = Ref<double>::D(qx, ax) * by * bz * sg.s[0];
    gt[e * DIM + 1] = bx * Ref<double>::D(qy, ay) * bz * sg.s[1];
    if (DIM == 3) gt[e * DIM + 2] = bx * by * Ref<double>::D(qz, az) * sg.s[2];
  }
  __syncthreads();
  for (int e = tid; e < TB::n_gt; e += nt) tab[e] = RealOps<R>::from(gt[e]);
  for (int e = tid; e < TB::n_wpsi; e += nt) tab[TB::n_gt + e] = RealOps<R>::from(wpsi[e]);
  for (int e = tid; e < NPR * DIM * NB; e += nt) {
    const int p = e / (DIM * NB), al = (e / NB) % DIM, a = e % NB;
    double acc = 0.0;
    for (int q = 0; q < NB; ++q) acc += wpsi[p * NB + q] * gt[(q * NB + a) * DIM + al];
    tab[TB::n_gt + TB::n_wpsi + e] = RealOps<R>::from(-acc);
  }
}

template <int DIM, bool TENSOR, typename R>
__global__ void __launch_bounds__(SetupCfg<DIM, TENSOR>::THREADS, TENSOR ? 2 : (std::is_same<R, DF64>::value ? 4 : 3))
k_patch_setup(Geom g, double gamma_d, SetupGeo sg, const R* __restrict__ tab, const double* __restrict__ coef,
              double* __restrict__ inv64, int pstride, DevStatus* st,
              const double* __restrict__ winv) {
  using C = SetupCfg<DIM, TENSOR>;
  using O = RealOps<R>;
  using TB = SetupTab<DIM>;
  constexpr int NP = C::NP, NB = C::NB, NPR = C::NPR, NM = C::NM, NC = C::NC, NSUB = C::NSUB;
  extern __shared__ double sm_raw[];
  __shared__ R s_winv[NPR * NPR];
  R* sm = reinterpret_cast<R*>(sm_raw);
  R* M = sm;                         // packed upper triangle of the patch matrix, swept in place
  R* pk = M + C::n_M;                // pivot column of the current sweep
  R* qk = pk + C::n_pk;              // pivot column / pivot
  R* gt = qk + C::n_qk;              // [q][a][k] physical gradient of phi_a at point q
  R* bt = gt + C::n_gt;              // [p][alpha][a]: B_K entries, -(psi_p, d phi_a / d x_alpha)_K
  R* wq = bt + C::n_bt;              // [q] |J| w_q mu_q, or [q][NC] |J| w_q C_q, of the current cell
  R* wpsi = wq + C::n_wq;            // [p][q] |J| w_q psi_p(q)
  R* T = wpsi + C::n_wpsi;           // tensor: [q][j][be][m] = (C_q eps(phi_b(j) e_be))_m
  unsigned char* rowof = reinterpret_cast<unsigned char*>(sm_raw + C::n_dbl);   // row of every packed entry
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long v = blockIdx.x;
  int vx, vy, vz;
  vertex_coords<DIM>(g, v, vx, vy, vz);
  const R zero = O::from(0.0), one = O::from(1.0), three = O::from(3.0);
  const R gamma = O::from(gamma_d), gvol = O::from(sg.gvol), ir2 = O::from(0.70710678118654752440);

  for (int e = tid; e < C::NPK; e += nt) M[e] = zero;
  for (int i = tid; i < NP; i += nt)
    for (int j = i; j < NP; ++j) rowof[tri_row(NP, i) + (j - i)] = (unsigned char)i;
  for (int e = tid; e < TB::n_gt; e += nt) gt[e] = tab[e];
  for (int e = tid; e < TB::n_wpsi; e += nt) wpsi[e] = tab[TB::n_gt + e];
  for (int e = tid; e < TB::n_bt; e += nt) bt[e] = tab[TB::n_gt + TB::n_wpsi + e];

  // contributions of the 2^d cells of the star
  for (int sc = 0; sc < NSUB; ++sc) {
    const int sx = sc & 1, sy = (sc >> 1) & 1, sz = (sc >> 2) & 1;
    const int cx = vx - 1 + sx, cy = vy - 1 + sy, cz = DIM == 3 ? vz - 1 + sz : 0;
    const bool valid = cx >= 0 && cx < g.n[0] && cy >= 0 && cy < g.n[1] &&
                       (DIM == 2 || (cz >= 0 && cz < g.n[2]));
    __syncthreads();
    if (!valid) continue;
    const long long cell = (long long)cx + (long long)g.n[0] * ((long long)cy + (long long)g.n[1] * cz);
    for (int e = tid; e < C::n_wq; e += nt) wq[e] = wpsi[TENSOR ? e / NC : e] * O::from(coef[cell * C::n_wq + e]);
    if (winv)
      for (int e = tid; e < NPR * NPR; e += nt) s_winv[e] = O::from(winv[cell * NPR * NPR + e]);
    __syncthreads();
    if constexpr (TENSOR) {
      // T[q][j][be] = C_q eps(phi_b e_be), b the cell-local node of sub-node j
      for (int e = tid; e < NB * NSUB * DIM; e += nt) {
        const int q = e / (NSUB * DIM), j = (e / DIM) % NSUB, be = e % DIM;
        int Q, b;
        sub_node<DIM>(j, sx, sy, sz, Q, b);
        // eps(phi_b e_be) in Mandel form has d nonzeros: slot be and the shear slots
        int n_[3];
        R e_[3];
        strain_nonzeros<DIM>(be, gt + (q * NB + b) * DIM, ir2, n_, e_);
        const R* Cq = wq + q * NC;
        R* t = T + e * NM;
        for (int m = 0; m < NM; ++m) {
          R acc = zero;
#pragma unroll
          for (int r = 0; r < DIM; ++r) {
            const int n = n_[r], lo = m < n ? m : n, hi = m < n ? n : m;
            acc = O::add_prod(acc, Cq[lo * NM - (lo * (lo - 1)) / 2 + (hi - lo)], e_[r]);
          }
          t[m] = acc;
        }
      }
      __syncthreads();
    }
    // Sub-node pairs i <= j (the pair (j, i) is the transpose): one thread per pair
    // (scalar mu: the d x d block from the 3x3 gradient products) or per (pair, row
    // component al) (tensor: d rows of products with T).  Entries go to
    // (min(row, col), max(row, col)); in a diagonal block (i == j) only row <= col.
    // (only the NSUB (NSUB + 1) / 2 pairs i <= j are enumerated, so no thread idles on i > j)
    constexpr int NAL = TENSOR ? DIM : 1;
    constexpr int NPAIR = NSUB * (NSUB + 1) / 2;
    for (int it = tid; it < NPAIR * NAL; it += nt) {
      const int pr = it / NAL, al0 = it % NAL;
      int i = 0, j = pr;
      while (j >= NSUB - i) { j -= NSUB - i; ++i; }
      j += i;
      int P, a, Q, b;
      sub_node<DIM>(i, sx, sy, sz, P, a);
      sub_node<DIM>(j, sx, sy, sz, Q, b);
      long long ndP, ndQ;
      if (!patch_node<DIM>(g, vx, vy, vz, P, ndP) || !patch_node<DIM>(g, vx, vy, vz, Q, ndQ)) continue;
      R V[DIM][DIM];
#pragma unroll
      for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int l = 0; l < DIM; ++l) V[k][l] = zero;
      if constexpr (!TENSOR) {
        // 2 mu eps(phi_b e_be) : eps(phi_a e_al) = mu (d_be phi_a d_al phi_b + delta_(al,be) grad phi_a . grad phi_b)
        R G[DIM][DIM];
#pragma unroll
        for (int k = 0; k < DIM; ++k)
#pragma unroll
          for (int l = 0; l < DIM; ++l) G[k][l] = zero;
        for (int q = 0; q < NB; ++q) {
          const R w = wq[q];
          const R* ga = gt + (q * NB + a) * DIM;
          const R* gb = gt + (q * NB + b) * DIM;
#pragma unroll
          for (int k = 0; k < DIM; ++k) {
            const R wa = w * ga[k];
#pragma unroll
            for (int l = 0; l < DIM; ++l) G[k][l] = O::add_prod(G[k][l], wa, gb[l]);
          }
        }
        R tr = zero;
#pragma unroll
        for (int k = 0; k < DIM; ++k) tr = O::add(tr, G[k][k]);
#pragma unroll
        for (int al = 0; al < DIM; ++al)
#pragma unroll
          for (int be = 0; be < DIM; ++be) V[al][be] = al == be ? O::add(G[be][al], tr) : G[be][al];
      } else {
        // (C eps(phi_b e_be)) : eps(phi_a e_al) with the d nonzeros of eps(phi_a e_al)
        for (int q = 0; q < NB; ++q) {
          int n_[3];
          R e_[3];
          strain_nonzeros<DIM>(al0, gt + (q * NB + a) * DIM, ir2, n_, e_);
          const R* t = T + (q * NSUB + j) * DIM * NM;
#pragma unroll
          for (int be = 0; be < DIM; ++be) {
            R acc = zero;
#pragma unroll
            for (int r = 0; r < DIM; ++r) acc = O::add_prod(acc, e_[r], t[be * NM + n_[r]]);
            V[al0][be] = O::add(V[al0][be], acc);
          }
        }
      }
#pragma unroll
      for (int al = 0; al < DIM; ++al) {
        if (TENSOR && al != al0) continue;
#pragma unroll
        for (int be = 0; be < DIM; ++be) {
          const int row = al * NB + P, col = be * NB + Q;
          if (i == j && row > col) continue;   // the diagonal block: upper triangle only
          R alv = zero, val = V[al][be];
          if (winv) {   // gamma B_K^T W_K^-1 B_K with W = M_p(1/mu)
            for (int p = 0; p < NPR; ++p)
              for (int p2 = 0; p2 < NPR; ++p2)
                alv = O::add_prod(alv, bt[(p * DIM + al) * NB + a] * s_winv[p * NPR + p2], bt[(p2 * DIM + be) * NB + b]);
            val = O::add_prod(val, gamma, alv);
          } else {      // W = M_p = |K| diag(1, 1/3, ..)
            for (int p = 0; p < NPR; ++p)
              alv = O::add_prod(alv, (p == 0 ? one : three) * bt[(p * DIM + al) * NB + a], bt[(p * DIM + be) * NB + b]);
            val = O::add_prod(val, gvol, alv);
          }
          const int lo = row < col ? row : col, hi = row < col ? col : row;
          M[tri_row(NP, lo) + (hi - lo)] = O::add(M[tri_row(NP, lo) + (hi - lo)], val);
        }
      }
    }
  }
  __syncthreads();
  // identity rows for nodes outside the domain or on the Dirichlet boundary
  for (int i = tid; i < NP; i += nt) {
    long long nd;
    if (!patch_node<DIM>(g, vx, vy, vz, i % NB, nd)) M[tri_row(NP, i)] = one;
  }
  __syncthreads();

  // symmetric sweep of every pivot in order: M -> -A_v^-1.  Two phases per pivot:
  // threads i < NP read the pivot column, form 1/pivot themselves (no wait on one
  // thread) and the scaled column; then every thread updates its contiguous segment
  // of the packed entries (row and column tracked incrementally), and threads i < NP
  // write the pivot row/column (entries the update skips).
  constexpr int SEG = (C::NPK + C::THREADS - 1) / C::THREADS;
  const int e0 = tid * SEG < C::NPK ? tid * SEG : C::NPK;
  const int e1 = e0 + SEG < C::NPK ? e0 + SEG : C::NPK;
  const int i0 = e0 < C::NPK ? (int)rowof[e0] : NP;
  const int j0 = e0 < C::NPK ? e0 - tri_row(NP, i0) + i0 : NP;
  for (int k = 0; k < NP; ++k) {
    R dinv = zero;
    if (tid < NP) {
      R d = M[tri_row(NP, k)];
      if (!(d > 0.f)) {
        if (tid == 0) report(st, 4 /* ALS_ENOTSPD */, v);
        d = one;
      }
      dinv = one / d;
      const int i = tid;
      const R p = (i == k) ? zero : M[i < k ? tri_row(NP, i) + (k - i) : tri_row(NP, k) + (i - k)];
      pk[i] = p;
      qk[i] = p * dinv;
    }
    __syncthreads();
    {
      int i = i0, j = j0;
      R qi = i < NP ? qk[i] : zero;
      for (int e = e0; e < e1; ++e) {
        if (i != k && j != k) M[e] = O::sub_prod(M[e], qi, pk[j]);
        if (++j == NP) {
          ++i;
          j = i;
          if (i < NP) qi = qk[i];
        }
      }
    }
    if (tid < NP) {
      const int i = tid;
      if (i == k) M[tri_row(NP, k)] = -dinv;
      else M[i < k ? tri_row(NP, i) + (k - i) : tri_row(NP, k) + (i - k)] = qk[i];
    }
    __syncthreads();
  }
  // A_v^-1 = -M, packed by diagonals in FP64 (the FP32 copies are derived from it)
  for (int e = tid; e < C::NPK; e += nt) {
    int t = 0;
    while (diag_start(NP, t + 1) <= e) ++t;
    const int i = e - diag_start(NP, t);
    inv64[v * pstride + e] = O::to_double(-M[tri_row(NP, i) + t]);
  }
}
