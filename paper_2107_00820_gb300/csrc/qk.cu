// The higher-order discretisation of the paper's Table k (Sec. 5.2.2): [Q3]^2 x P2^disc
// on uniform quad meshes, FP64 and FP32, the whole hot path -- A_gamma / Stokes operator
// applies, vertex-star patch setup and smoother, robust transfers, coarse images, mass and
// Schur blocks -- so that the context's multigrid cycle and FGMRES run on it unchanged.
//
// Velocity: continuous Q3, nodal basis on the 4 equispaced nodes -1, -1/3, 1/3, 1 per
// axis and cell, node lattice 3n + 1 per direction, x fastest.  Pressure: discontinuous
// P2, the monomials xi^a eta^b (a + b <= 2) in reference coordinates, ordered by total
// degree, xi before eta: {1, xi, eta, xi^2, xi eta, eta^2}; 6 per cell.  Quadrature:
// 4 x 4 Gauss-Legendre points per cell.  Vertex stars: the free nodes at lattice offsets
// -2..2 from 3v in each direction (5 x 5 nodes, 50 dofs at an interior vertex); the
// interior of a coarse cell is the star of the fine vertex at its centre (Eq. (Ptilde)).
// Deterministic: per-cell and per-star outputs are staged and summed per node in a
// fixed order.
#include <math.h>

#include <type_traits>

#include "cell.cuh"
#include "krylov.h"
#include "level.h"
#include "qk_tables.h"

namespace als {
namespace qk {

constexpr int K = 3;           // polynomial order
constexpr int N1 = K + 1;      // nodes (and Gauss points) per axis and cell
constexpr int NB = N1 * N1;    // nodes per cell
constexpr int NQ = NB;         // Gauss points per cell
constexpr int NE = 2 * NB;     // velocity dofs per cell
constexpr int NPR = 6;         // pressure monomials per cell
constexpr int S1 = 2 * K - 1;  // star nodes per axis
constexpr int NS = 2 * S1 * S1;   // star dofs (50)
// FP32 star storage in wrapped rows W_t[i] = A(i, (i + t) mod NS), t = 0..NS/2 (NS is even:
// row NS/2 holds each pair {i, i + NS/2} twice, and the product reads it once per row), rows
// padded to 52 entries (16-byte rows): 1,352 floats a star against 1,276 for the packed
// diagonals; the product then needs no per-entry choice of diagonal
constexpr int kWT = NS / 2 + 1;   // 26
constexpr int kWLD = 52;
constexpr int kWStride = kWT * kWLD;
static_assert(NS % 2 == 0 && kWLD % 4 == 0 && kWLD >= NS, "wrapped-row layout");

// 1D tables at the Gauss points: L[q][a] = l_a(g_q), D[q][a] = l_a'(g_q), W[q]; the 2D
// pressure monomials at the points PSI[q][p]; the prolongation weights PW[f][a] = l_a(xi_f)
// at xi_f = f / 3 - 1, f = 0..6 (the fine nodes of a coarse cell per axis)
__constant__ double cL[N1][N1], cD[N1][N1], cW[N1], cPSI[NQ][NPR], cPW[2 * K + 1][N1];
// the FP32 cycle's copies (an FP64 operation, a conversion included, costs ~70 FP32 ones
// on this GPU) and the 2D point weights w_qx w_qy in both precisions
__constant__ float cLf[N1][N1], cDf[N1][N1], cPSIf[NQ][NPR], cPWf[2 * K + 1][N1], cW2f[NQ];
__constant__ double cW2[NQ];
template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ double L(int q, int a) { return cL[q][a]; }
  static __device__ __forceinline__ double D(int q, int a) { return cD[q][a]; }
  static __device__ __forceinline__ double psi(int q, int p) { return cPSI[q][p]; }
  static __device__ __forceinline__ double pw(int f, int a) { return cPW[f][a]; }
  static __device__ __forceinline__ double w2(int q) { return cW2[q]; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ float L(int q, int a) { return cLf[q][a]; }
  static __device__ __forceinline__ float D(int q, int a) { return cDf[q][a]; }
  static __device__ __forceinline__ float psi(int q, int p) { return cPSIf[q][p]; }
  static __device__ __forceinline__ float pw(int f, int a) { return cPWf[f][a]; }
  static __device__ __forceinline__ float w2(int q) { return cW2f[q]; }
};
// per-level scalars of the cell kernel in its precision, formed on the host
template <typename T>
struct CellScal {
  T sx, sy, wdet, gamma;
};
template <typename T>
static CellScal<T> cell_scal(const Geom& g, double gamma) {
  return CellScal<T>{(T)(2.0 / g.h[0]), (T)(2.0 / g.h[1]), (T)(0.25 * g.h[0] * g.h[1]), (T)gamma};
}

static void host_tables(double L[N1][N1], double D[N1][N1], double W[N1], double PSI[NQ][NPR],
                        double PW[2 * K + 1][N1]) {
  double g[N1];
  qk_tab::tables_1d(g, L, D, W, PW);
  const int ex[NPR][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
  for (int q = 0; q < NQ; ++q) {
    const double xi = g[q % N1], eta = g[q / N1];
    for (int p = 0; p < NPR; ++p) PSI[q][p] = pow(xi, ex[p][0]) * pow(eta, ex[p][1]);
  }
}

// uploaded once per process (before any context of order 3 captures a cycle)
void ensure_tables() {
  static bool done = false;
  if (done) return;
  double L[N1][N1], D[N1][N1], W[N1], PSI[NQ][NPR], PW[2 * K + 1][N1];
  host_tables(L, D, W, PSI, PW);
  cudaMemcpyToSymbol(cL, L, sizeof(L));
  cudaMemcpyToSymbol(cD, D, sizeof(D));
  cudaMemcpyToSymbol(cW, W, sizeof(W));
  cudaMemcpyToSymbol(cPSI, PSI, sizeof(PSI));
  cudaMemcpyToSymbol(cPW, PW, sizeof(PW));
  float Lf[N1][N1], Df[N1][N1], PSIf[NQ][NPR], PWf[2 * K + 1][N1], W2f[NQ];
  double W2[NQ];
  for (int q = 0; q < N1; ++q)
    for (int a = 0; a < N1; ++a) { Lf[q][a] = (float)L[q][a]; Df[q][a] = (float)D[q][a]; }
  for (int q = 0; q < NQ; ++q) {
    for (int p = 0; p < NPR; ++p) PSIf[q][p] = (float)PSI[q][p];
    W2[q] = W[q % N1] * W[q / N1];
    W2f[q] = (float)W2[q];
  }
  for (int f = 0; f <= 2 * K; ++f)
    for (int a = 0; a < N1; ++a) PWf[f][a] = (float)PW[f][a];
  cudaMemcpyToSymbol(cLf, Lf, sizeof(Lf));
  cudaMemcpyToSymbol(cDf, Df, sizeof(Df));
  cudaMemcpyToSymbol(cPSIf, PSIf, sizeof(PSIf));
  cudaMemcpyToSymbol(cPWf, PWf, sizeof(PWf));
  cudaMemcpyToSymbol(cW2f, W2f, sizeof(W2f));
  cudaMemcpyToSymbol(cW2, W2, sizeof(W2));
  done = true;
}

// The tables in shared memory, in precision T: lanes index them by their own point or node,
// which the constant cache would serialise.  wq = the quadrature weight times |J|;
// gx, gy = the physical derivatives of every node basis at every point.
template <typename T>
struct SharedTables {
  T gx[NQ][NB], gy[NQ][NB], wq[NQ], psi[NQ][NPR];
};
template <typename T>
__device__ __forceinline__ void load_tables(SharedTables<T>& t, T sx, T sy, T wdet) {
  for (int e = threadIdx.x; e < NQ * NB; e += blockDim.x) {
    const int q = e / NB, a = e % NB, qx = q % N1, qy = q / N1, ax = a % N1, ay = a / N1;
    t.gx[q][a] = Tab<T>::D(qx, ax) * Tab<T>::L(qy, ay) * sx;
    t.gy[q][a] = Tab<T>::L(qx, ax) * Tab<T>::D(qy, ay) * sy;
  }
  for (int e = threadIdx.x; e < NQ * NPR; e += blockDim.x) t.psi[e / NPR][e % NPR] = Tab<T>::psi(e / NPR, e % NPR);
  for (int q = threadIdx.x; q < NQ; q += blockDim.x) t.wq[q] = Tab<T>::w2(q) * wdet;
  __syncthreads();
}
__device__ __forceinline__ double phi(int q, int a) { return cL[q % N1][a % N1] * cL[q / N1][a / N1]; }

// ---------------------------------------------------------------------------
// operator apply: one warp per cell, lanes 0..15 = Gauss points, then = nodes
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_qk_cells(Geom g, CellScal<T> cs, const T* __restrict__ x, const T* __restrict__ mu,
                                                  const T* __restrict__ winv, const T* __restrict__ p_in,
                                                  T* __restrict__ p_out, T* __restrict__ ebuf) {
  constexpr bool RAW = (MODE & OP_RAW) != 0, VISC = (MODE & OP_VISC) != 0, AL = (MODE & OP_AL) != 0;
  constexpr bool BT = (MODE & OP_BT) != 0, BO = (MODE & OP_B) != 0;
  constexpr bool NEED_U = VISC || AL || BO, NEED_FLUX = VISC || AL || BT;
  __shared__ SharedTables<T> tb;
  __shared__ T us[8][2][NB];
  __shared__ T ss[8][NQ][4];
  load_tables<T>(tb, cs.sx, cs.sy, cs.wdet);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long cell = (long long)blockIdx.x * 8 + w;
  if (cell >= g.ncells) return;
  const int cx = (int)(cell % g.n[0]), cy = (int)(cell / g.n[0]);
  if (lane < NB) {
    const int i = K * cx + lane % N1, j = K * cy + lane / N1;
    const bool bnd = i == 0 || i == g.nn[0] - 1 || j == 0 || j == g.nn[1] - 1;
    const long long nd = (long long)i + (long long)g.nn[0] * j;
    for (int c = 0; c < 2; ++c) us[w][c][lane] = (NEED_U && (RAW || !bnd)) ? x[c * g.N + nd] : T(0);
  }
  __syncwarp();
  const int q = lane < NQ ? lane : 0;
  T G00 = T(0), G01 = T(0), G10 = T(0), G11 = T(0);
  if (NEED_U && lane < NQ) {
#pragma unroll 4
    for (int a = 0; a < NB; ++a) {
      const T dx = tb.gx[q][a], dy = tb.gy[q][a], u0 = us[w][0][a], u1 = us[w][1][a];
      G00 += u0 * dx;
      G01 += u0 * dy;
      G10 += u1 * dx;
      G11 += u1 * dy;
    }
  }
  const T div = G00 + G11;
  T P = T(0);   // the pressure-like field at the point: gamma pi + p_in
  if (AL || BO) {
    T bu[NPR];   // (B u)_p = -sum_q w |J| psi_p div u
#pragma unroll
    for (int p = 0; p < NPR; ++p) {
      T v = lane < NQ ? -tb.wq[q] * tb.psi[q][p] * div : T(0);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      bu[p] = v;
    }
    if (BO && lane == 0)
      for (int p = 0; p < NPR; ++p) p_out[cell * NPR + p] = bu[p];
    if (AL && lane < NQ) {
      const T* Wc = winv + cell * NPR * NPR;
      T pi = T(0);
#pragma unroll
      for (int p = 0; p < NPR; ++p) {
        T sp = T(0);
#pragma unroll
        for (int r = 0; r < NPR; ++r) sp += Wc[p * NPR + r] * bu[r];
        pi += tb.psi[q][p] * sp;
      }
      P += cs.gamma * pi;
    }
  }
  if (BT && lane < NQ)
    for (int p = 0; p < NPR; ++p) P += tb.psi[q][p] * p_in[cell * NPR + p];
  if (!NEED_FLUX) return;
  if (lane < NQ) {
    const T m2 = VISC ? T(2) * mu[cell * NQ + q] : T(0);
    const T e01 = T(0.5) * (G01 + G10);
    const T wq = tb.wq[q];
    ss[w][q][0] = wq * (m2 * G00 - P);
    ss[w][q][1] = wq * (m2 * e01);
    ss[w][q][2] = wq * (m2 * e01);
    ss[w][q][3] = wq * (m2 * G11 - P);
  }
  __syncwarp();
  if (lane < NB) {
    const int a = lane;
    T y0 = T(0), y1 = T(0);
#pragma unroll 4
    for (int qq = 0; qq < NQ; ++qq) {
      const T dx = tb.gx[qq][a], dy = tb.gy[qq][a];
      y0 += ss[w][qq][0] * dx + ss[w][qq][1] * dy;
      y1 += ss[w][qq][2] * dx + ss[w][qq][3] * dy;
    }
    ebuf[(cell * 2 + 0) * NB + a] = y0;
    ebuf[(cell * 2 + 1) * NB + a] = y1;
  }
}

// the cells (and local index) containing lattice index i along an axis of n cells
__device__ __forceinline__ int cells_of(int i, int n, int (&c)[2], int (&a)[2]) {
  int m = 0;
  const int c0 = i / K, r = i - K * c0;
  if (r == 0 && c0 > 0) { c[m] = c0 - 1; a[m] = K; ++m; }
  if (c0 < n) { c[m] = c0; a[m] = r; ++m; }
  return m;
}

// y(node) = sum of the staged cell outputs of the cells containing it, fixed order;
// keep_bnd: y = x at Dirichlet nodes; raw: no Dirichlet treatment
template <typename T>
__device__ __forceinline__ T qk_gather_value(const Geom& g, const T* __restrict__ ebuf, const T* __restrict__ x,
                                             long long t, int keep_bnd, int raw) {
  const int comp = (int)(t / g.N);
  const long long nd = t - comp * g.N;
  const int i = (int)(nd % g.nn[0]), j = (int)(nd / g.nn[0]);
  const bool bnd = i == 0 || i == g.nn[0] - 1 || j == 0 || j == g.nn[1] - 1;
  if (bnd && !raw) return keep_bnd ? x[t] : T(0);
  int cxs[2], axs[2], cys[2], ays[2];
  const int mx = cells_of(i, g.n[0], cxs, axs), my = cells_of(j, g.n[1], cys, ays);
  T acc = T(0);
  for (int b = 0; b < my; ++b)
    for (int a = 0; a < mx; ++a) {
      const long long cell = (long long)cxs[a] + (long long)g.n[0] * cys[b];
      acc += ebuf[(cell * 2 + comp) * NB + axs[a] + N1 * ays[b]];
    }
  return acc;
}

template <typename T>
__global__ void k_qk_gather(Geom g, const T* __restrict__ ebuf, const T* __restrict__ x, T* __restrict__ y, int keep_bnd,
                            int raw) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.N) return;
  y[t] = qk_gather_value<T>(g, ebuf, x, t, keep_bnd, raw);
}

// The gather fused with the reduction that consumes its result, as for order 2 (the
// GMRES smoother's Arnoldi step): y = b + sigma A x (b NULL: sigma A x; Dirichlet rows of
// A x are x, the identity);  start = 0: out[j] = (V_j . y) / hn[j], j < k;  start = 1:
// |y|^2 starts the GMRES cycle.  Block partials in a fixed order: reproducible.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_qk_gather_epi(Geom g, const T* __restrict__ ebuf,
                                                               const T* __restrict__ x, T* __restrict__ y,
                                                               const T* __restrict__ b, double sigma, int k,
                                                               const T* __restrict__ V, long long ld,
                                                               T* __restrict__ out, int start, GmresDev sd,
                                                               double* __restrict__ partial) {
  __shared__ T nrm2_s[1];
  const GmresView<T> st = gmres_view<T>(sd);
  T* rows = reinterpret_cast<T*>(partial + 1);
  const int kk = start ? 1 : k;
  T acc[KMAXB];
#pragma unroll
  for (int jj = 0; jj < KMAXB; ++jj) acc[jj] = T(0);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < 2 * g.N) {
    const T v = (b ? b[t] : T(0)) + (T)sigma * qk_gather_value<T>(g, ebuf, x, t, 1, 0);
    y[t] = v;
    if (start) {
      acc[0] = v * v;
    } else {
#pragma unroll
      for (int jj = 0; jj < KMAXB; ++jj)
        if (jj < k) acc[jj] = V[(long long)jj * ld + t] * v;
    }
  }
  block_partials<T, T>(acc, kk, rows + (long long)blockIdx.x * kk);
  if (last_block(partial)) {
    if (start) {
      finish_sums<T>(partial, 1, nrm2_s);
      if (threadIdx.x == 0) gmres_start(st, nrm2_s[0]);
    } else {
      finish_sums<T>(partial, k, out, st.hn);
    }
  }
}

template <typename T, int MODE>
static void apply_mode(const LevelDev& L, double gamma, const void* x, void* y, const void* p_in, void* p_out,
                       cudaStream_t s) {
  constexpr bool NEED_FLUX = (MODE & (OP_VISC | OP_AL | OP_BT)) != 0;
  const T* mu = std::is_same<T, double>::value ? (const T*)L.coef64 : (const T*)L.coef32;
  const T* winv = std::is_same<T, double>::value ? (const T*)L.winv64 : (const T*)L.winv32;
  k_qk_cells<T, MODE><<<(unsigned)((L.g.ncells + 7) / 8), 256, 0, s>>>(L.g, cell_scal<T>(L.g, gamma), (const T*)x, mu, winv,
                                                                      (const T*)p_in, (T*)p_out, (T*)L.ebuf);
  if (NEED_FLUX) {
    const int keep = ((MODE & OP_VISC) && !(MODE & OP_RAW)) ? 1 : 0;
    k_qk_gather<T><<<(unsigned)((2 * L.g.N + 255) / 256), 256, 0, s>>>(L.g, (const T*)L.ebuf, (const T*)x, (T*)y,
                                                                        keep, (MODE & OP_RAW) ? 1 : 0);
  }
  count_launch(NEED_FLUX ? 2 : 1);
}

template <typename T>
static void apply_t(const LevelDev& L, int mode, double gamma, const void* x, void* y, const void* p_in, void* p_out,
                    cudaStream_t s) {
  switch (mode) {
    case OP_VISC | OP_AL: apply_mode<T, OP_VISC | OP_AL>(L, gamma, x, y, p_in, p_out, s); break;
    case OP_AL: apply_mode<T, OP_AL>(L, gamma, x, y, p_in, p_out, s); break;
    case OP_B: apply_mode<T, OP_B>(L, gamma, x, y, p_in, p_out, s); break;
    case OP_BT: apply_mode<T, OP_BT>(L, gamma, x, y, p_in, p_out, s); break;
    case OP_VISC | OP_AL | OP_BT | OP_B: apply_mode<T, OP_VISC | OP_AL | OP_BT | OP_B>(L, gamma, x, y, p_in, p_out, s); break;
    case OP_VISC | OP_AL | OP_RAW: apply_mode<T, OP_VISC | OP_AL | OP_RAW>(L, gamma, x, y, p_in, p_out, s); break;
    case OP_B | OP_RAW: apply_mode<T, OP_B | OP_RAW>(L, gamma, x, y, p_in, p_out, s); break;
    default: break;
  }
}

// F_(c,a) = sum_q |J| w_q f_c(x_q) phi_a(x_q), staged per cell, summed per node
__global__ void k_qk_load(Geom g, const double* __restrict__ f, double* __restrict__ ebuf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ncells * NE) return;
  const long long cell = t / NE;
  const int e = (int)(t % NE), comp = e / NB, a = e % NB;
  const double wdet = 0.25 * g.h[0] * g.h[1];
  double acc = 0.0;
  for (int q = 0; q < NQ; ++q) acc += cW[q % N1] * cW[q / N1] * wdet * f[(cell * NQ + q) * 2 + comp] * phi(q, a);
  ebuf[(cell * 2 + comp) * NB + a] = acc;
}

// ---------------------------------------------------------------------------
// per-cell mass blocks: M_K(1/mu)^-1 and M_K^-1 (6 x 6, Gauss-Jordan), the augmentation
// weight's inverse W^-1 (W = M_p or M_p(1/mu)) and the Schur blocks S of Eq. (P1P2):
// P1: M_K(1/mu)^-1 + gamma M_K^-1, P2: (1 + gamma) M_K(1/mu)^-1.  One thread per cell.
// ---------------------------------------------------------------------------
__device__ void inv6(double (&A)[NPR][NPR], DevStatus* st, long long where) {
  double Iv[NPR][NPR];
  for (int i = 0; i < NPR; ++i)
    for (int j = 0; j < NPR; ++j) Iv[i][j] = i == j ? 1.0 : 0.0;
  for (int k = 0; k < NPR; ++k) {
    const double pv = A[k][k];
    if (!(pv > 0.0)) { report(st, 4 /* ALS_ENOTSPD */, where); return; }
    const double ip = 1.0 / pv;
    for (int j = 0; j < NPR; ++j) { A[k][j] *= ip; Iv[k][j] *= ip; }
    for (int i = 0; i < NPR; ++i) {
      if (i == k) continue;
      const double f = A[i][k];
      for (int j = 0; j < NPR; ++j) { A[i][j] -= f * A[k][j]; Iv[i][j] -= f * Iv[k][j]; }
    }
  }
  for (int i = 0; i < NPR; ++i)
    for (int j = 0; j < NPR; ++j) A[i][j] = Iv[i][j];
}

__global__ void k_qk_mass(Geom g, double gamma, const double* __restrict__ mu, int w_mu, int variant,
                          double* __restrict__ winv64, float* __restrict__ winv32, double* __restrict__ S, DevStatus* st) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= g.ncells) return;
  const double wdet = 0.25 * g.h[0] * g.h[1];
  double Mm[NPR][NPR], M[NPR][NPR];
  for (int p = 0; p < NPR; ++p)
    for (int r = 0; r < NPR; ++r) { Mm[p][r] = 0.0; M[p][r] = 0.0; }
  for (int q = 0; q < NQ; ++q) {
    const double wq = cW[q % N1] * cW[q / N1] * wdet;
    const double im = 1.0 / mu[cell * NQ + q];
    for (int p = 0; p < NPR; ++p)
      for (int r = 0; r < NPR; ++r) {
        M[p][r] += wq * cPSI[q][p] * cPSI[q][r];
        Mm[p][r] += wq * im * cPSI[q][p] * cPSI[q][r];
      }
  }
  inv6(Mm, st, cell);
  inv6(M, st, cell);
  for (int p = 0; p < NPR; ++p)
    for (int r = 0; r < NPR; ++r) {
      const double wv = w_mu ? Mm[p][r] : M[p][r];
      if (winv64) winv64[cell * NPR * NPR + p * NPR + r] = wv;
      if (winv32) winv32[cell * NPR * NPR + p * NPR + r] = (float)wv;
      if (S) S[cell * NPR * NPR + p * NPR + r] = variant == 0 ? Mm[p][r] + gamma * M[p][r] : (1.0 + gamma) * Mm[p][r];
    }
}

// ---------------------------------------------------------------------------
// vertex stars: setup (assembly from the star's cells, Gauss-Jordan inversion in shared
// memory, FP64 packed-by-diagonals and its FP32 rounding), products, node gather
// ---------------------------------------------------------------------------
// star entry e = comp * 25 + (ox + 2) + 5 (oy + 2) of vertex v: node (3 vx + ox, 3 vy + oy)
__device__ __forceinline__ bool star_node(const Geom& g, int vx, int vy, int e, long long& nd) {
  const int o = e % (S1 * S1), ox = o % S1 - (K - 1), oy = o / S1 - (K - 1);
  const int i = K * vx + ox, j = K * vy + oy;
  if (i <= 0 || i >= g.nn[0] - 1 || j <= 0 || j >= g.nn[1] - 1) return false;
  nd = (long long)i + (long long)g.nn[0] * j;
  return true;
}

__global__ void __launch_bounds__(256) k_qk_star_setup(Geom g, double gamma, const double* __restrict__ mu,
                                                       const double* __restrict__ winv, double* __restrict__ inv64,
                                                       float* __restrict__ inv32, int pstride, DevStatus* st) {
  __shared__ double M[NS][NS + 1];
  __shared__ double Ae[NE][NE + 1];
  __shared__ double Bm[NPR][NE], WB[NPR][NE];
  __shared__ double rowk[NS], colk[NS];
  __shared__ int s_bad;
  __shared__ SharedTables<double> tb;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long v = blockIdx.x;
  const int vx = (int)(v % (g.n[0] + 1)), vy = (int)(v / (g.n[0] + 1));
  load_tables<double>(tb, 2.0 / g.h[0], 2.0 / g.h[1], 0.25 * g.h[0] * g.h[1]);   // FP64 setup
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < NS * NS; e += nt) M[e / NS][e % NS] = 0.0;
  // B_K (the same on every cell): B[p][(c, a)] = -sum_q w |J| psi_p d_c phi_a
  for (int e = tid; e < NPR * NE; e += nt) {
    const int p = e / NE, c = (e % NE) / NB, a = e % NB;
    double acc = 0.0;
    for (int q = 0; q < NQ; ++q) acc -= tb.wq[q] * tb.psi[q][p] * (c == 0 ? tb.gx[q][a] : tb.gy[q][a]);
    Bm[p][e % NE] = acc;
  }
  __syncthreads();
  for (int cy = vy - 1; cy <= vy; ++cy)
    for (int cx = vx - 1; cx <= vx; ++cx) {
      if (cx < 0 || cy < 0 || cx >= g.n[0] || cy >= g.n[1]) continue;
      const long long cell = (long long)cx + (long long)g.n[0] * cy;
      const double* Wc = winv + cell * NPR * NPR;
      for (int e = tid; e < NPR * NE; e += nt) {   // W^-1 B
        const int p = e / NE, j = e % NE;
        double acc = 0.0;
        for (int r = 0; r < NPR; ++r) acc += Wc[p * NPR + r] * Bm[r][j];
        WB[p][j] = acc;
      }
      __syncthreads();
      // element A_gamma: 2 mu eps(phi_i) : eps(phi_j) + gamma B^T W^-1 B
      for (int e = tid; e < NE * NE; e += nt) {
        const int i = e / NE, j = e % NE, ci = i / NB, ai = i % NB, cj = j / NB, aj = j % NB;
        double acc = 0.0;
        for (int q = 0; q < NQ; ++q) {
          const double wq = tb.wq[q] * 2.0 * mu[cell * NQ + q];
          const double gi0 = tb.gx[q][ai], gi1 = tb.gy[q][ai];
          const double gj0 = tb.gx[q][aj], gj1 = tb.gy[q][aj];
          // eps(phi_i e_ci) : eps(phi_j e_cj) = (delta gi.gj + d_cj phi_i d_ci phi_j) / 2
          const double dot = (ci == cj ? gi0 * gj0 + gi1 * gj1 : 0.0) + (cj == 0 ? gi0 : gi1) * (ci == 0 ? gj0 : gj1);
          acc += wq * 0.5 * dot;
        }
        double al = 0.0;
        for (int p = 0; p < NPR; ++p) al += Bm[p][i] * WB[p][j];
        Ae[i][j] = acc + gamma * al;
      }
      __syncthreads();
      // scatter into the star matrix: element node (3cx + ax, 3cy + ay) at offset (.. - 3v)
      for (int e = tid; e < NE * NE; e += nt) {
        const int i = e / NE, j = e % NE, ci = i / NB, ai = i % NB, cj = j / NB, aj = j % NB;
        const int oxi = K * cx + ai % N1 - K * vx, oyi = K * cy + ai / N1 - K * vy;
        const int oxj = K * cx + aj % N1 - K * vx, oyj = K * cy + aj / N1 - K * vy;
        if (oxi < -(K - 1) || oxi > K - 1 || oyi < -(K - 1) || oyi > K - 1) continue;
        if (oxj < -(K - 1) || oxj > K - 1 || oyj < -(K - 1) || oyj > K - 1) continue;
        const int si = ci * S1 * S1 + (oxi + K - 1) + S1 * (oyi + K - 1);
        const int sj = cj * S1 * S1 + (oxj + K - 1) + S1 * (oyj + K - 1);
        M[si][sj] += Ae[i][j];
      }
      __syncthreads();
    }
  // identity rows and columns at absent and Dirichlet nodes
  for (int e = tid; e < NS * NS; e += nt) {
    const int i = e / NS, j = e % NS;
    long long nd;
    const bool fi = star_node(g, vx, vy, i % (S1 * S1), nd), fj = star_node(g, vx, vy, j % (S1 * S1), nd);
    if (!fi || !fj) M[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  // in-place Gauss-Jordan inversion (SPD: pivots are the Schur complements, no pivoting)
  for (int k = 0; k < NS; ++k) {
    const double pv = M[k][k];
    if (!(pv > 0.0)) {
      if (tid == 0 && !s_bad) { report(st, 4 /* ALS_ENOTSPD */, v); s_bad = 1; }
    }
    const double ip = pv > 0.0 ? 1.0 / pv : 1.0;
    if (tid < NS) {
      rowk[tid] = M[k][tid] * ip;
      colk[tid] = M[tid][k];
    }
    __syncthreads();
    for (int e = tid; e < NS * NS; e += nt) {
      const int i = e / NS, j = e % NS;
      if (i == k && j == k) M[i][j] = ip;
      else if (i == k) M[i][j] = rowk[j];
      else if (j == k) M[i][j] = -colk[i] * ip;
      else M[i][j] -= colk[i] * rowk[j];
    }
    __syncthreads();
  }
  // FP64: upper triangle by diagonals (entry (i, i+t)); FP32: the wrapped rows; both symmetrised
  for (int t = 0; t < NS; ++t) {
    const int base = diag_start(NS, t);
    for (int i = tid; i + t < NS; i += nt) inv64[v * pstride + base + i] = 0.5 * (M[i][i + t] + M[i + t][i]);
  }
  for (int e = tid; e < kWStride; e += nt) {
    const int t = e / kWLD, i = e % kWLD, j = i + t < NS ? i + t : i + t - NS;
    inv32[v * kWStride + e] = i < NS ? (float)(0.5 * (M[i][j] + M[j][i])) : 0.f;
  }
}

// y_v = A_v^-1 r|_v: one warp per star (vertex), entries by lanes, diagonals in order;
// interior: the stars of the fine vertices 2K+1 at the coarse-cell centres, written (mode 1)
// or subtracted (mode 2) straight into the nodes; else into the scratch rows [vertex][50].
// The warp first copies its star's packed inverse (pstride = 1276 entries) into shared
// memory with 16-byte loads from all lanes, all in flight at once, then forms the rows from
// there: one memory latency per star instead of one per diagonal.
constexpr int kStarStride = 1276;   // packed_stride(50)
template <typename T>
__host__ __device__ constexpr int star_warps() { return sizeof(T) == 4 ? 8 : 4; }   // 41 KB of shared memory a block

template <typename T>
__global__ void __launch_bounds__(32 * star_warps<T>()) k_qk_star_apply(Geom g, const T* __restrict__ inv, int pstride,
                                                                       int interior, int mode, const T* __restrict__ r,
                                                                       T* __restrict__ out) {
  constexpr int R = (NS + 31) / 32, WPB = star_warps<T>();
  constexpr int NV = kStarStride * (int)sizeof(T) / 16;   // 16-byte words of one star
  __shared__ T rs[WPB][NS];
  __shared__ uint4 sbuf[WPB][NV];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long count = interior ? (long long)(g.n[0] / 2) * (g.n[1] / 2) : (long long)(g.n[0] + 1) * (g.n[1] + 1);
  const long long item = (long long)blockIdx.x * WPB + w;
  if (item >= count || pstride != kStarStride) return;
  int vx, vy;
  if (interior) { vx = 2 * (int)(item % (g.n[0] / 2)) + 1; vy = 2 * (int)(item / (g.n[0] / 2)) + 1; }
  else { vx = (int)(item % (g.n[0] + 1)); vy = (int)(item / (g.n[0] + 1)); }
  const long long v = (long long)vx + (long long)(g.n[0] + 1) * vy;
  const uint4* src = reinterpret_cast<const uint4*>(inv + v * kStarStride);
#pragma unroll 4
  for (int e = lane; e < NV; e += 32) sbuf[w][e] = __ldg(src + e);
  for (int e = lane; e < NS; e += 32) {
    long long nd;
    rs[w][e] = star_node(g, vx, vy, e, nd) ? r[(e / (S1 * S1)) * g.N + nd] : T(0);
  }
  __syncwarp();
  T acc[R];
  for (int k = 0; k < R; ++k) acc[k] = T(0);
  // symmetric product over the wrapped diagonals: row i takes entry (i, (i + t) mod NS),
  // entry i of diagonal t while i + t < NS, else entry i + t - NS of diagonal NS - t (its
  // symmetric partner), so every lane of a row chunk multiplies at every t
  const T* S = reinterpret_cast<const T*>(&sbuf[w][0]);
#pragma unroll 5
  for (int t = 0; t < NS; ++t) {
    const T* du = S + diag_start(NS, t);
    const T* dl = S + (t > 0 ? diag_start(NS, NS - t) - (NS - t) : 0);
    for (int k = 0; k < R; ++k) {
      const int i = lane + 32 * k;
      if (i < NS) {
        const int j = i + t;
        const bool up = j < NS;
        acc[k] += (up ? du[i] : dl[i]) * rs[w][up ? j : j - NS];
      }
    }
  }
  for (int k = 0; k < R; ++k) {
    const int i = lane + 32 * k;
    if (i >= NS) continue;
    if (!interior) {
      out[v * NS + i] = acc[k];
    } else {
      long long nd;
      if (star_node(g, vx, vy, i, nd)) {
        T* o = out + (i / (S1 * S1)) * g.N + nd;
        *o = mode == 2 ? *o - acc[k] : acc[k];
      }
    }
  }
}

// The FP32 product from the wrapped rows, one star at a time per warp (8 warps a block), the
// star's rows staged in shared memory, r held twice over so that no index wraps;
// y_i = sum_(t <= NS/2) W_t[i] r_(i+t) + sum_(0 < t < NS/2) W_t[i-t] r_(i-t) (indices mod NS),
// rows i and i + NS/2 on one lane (see below).
// interior / mode as k_qk_star_apply.  Persistent: the host sizes the grid to
// kStarWBlocksPerSM blocks an SM and each warp walks the stars item, item + warps, ...;
// while it multiplies one star out of shared memory, the next star's rows (16-byte loads,
// at most eleven a lane) and r values are already on their way into registers, so every
// star but a warp's first has its memory latency hidden behind the previous star's
// products.  (With one star a warp and no prefetch, each star paid its dependent round
// trips in full: 7.7 long-scoreboard stalls per issued instruction, DRAM 35 % busy.)
// Outputs never overlap inputs within a launch (the scratch rows, or interior nodes of
// distinct coarse cells), so reading the next star's r early is safe.
constexpr int kStarWBlocksPerSM = 3;   // 3 x 256 threads at <= 85 registers, 3 x 46.5 KB shared

__global__ void __launch_bounds__(256, kStarWBlocksPerSM) k_qk_star_apply_w(Geom g, const float* __restrict__ inv,
                                                                            int interior, int mode,
                                                                            const float* __restrict__ r,
                                                                            float* __restrict__ out) {
  constexpr int R = (NS + 31) / 32, WPB = 8, NV = kWStride / 4, PF = (NV + 31) / 32, H = NS / 2;
  static_assert(H <= 32 && kWT == H + 1, "two rows a lane");
  __shared__ float rs2[WPB][2 * NS];
  __shared__ __align__(16) float ws[WPB][kWStride];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long count = interior ? (long long)(g.n[0] / 2) * (g.n[1] / 2) : (long long)(g.n[0] + 1) * (g.n[1] + 1);
  const long long nwarps = (long long)gridDim.x * WPB;
  long long item = (long long)blockIdx.x * WPB + w;
  if (item >= count) return;   // uniform over the warp; no block barrier below
  const auto vertex = [&](long long it, int& vx, int& vy) {
    if (interior) { vx = 2 * (int)(it % (g.n[0] / 2)) + 1; vy = 2 * (int)(it / (g.n[0] / 2)) + 1; }
    else { vx = (int)(it % (g.n[0] + 1)); vy = (int)(it / (g.n[0] + 1)); }
  };
  // a star's rows and r values into registers (consumed by the next pass's staging)
  float4 pw[PF];
  float pr[R];
  const auto fetch = [&](long long it) {
    int fx, fy;
    vertex(it, fx, fy);
    const float4* src = reinterpret_cast<const float4*>(inv + ((long long)fx + (long long)(g.n[0] + 1) * fy) * kWStride);
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = lane + 32 * q;
      if (e < NV) pw[q] = __ldg(src + e);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int e = lane + 32 * k;
      long long nd;
      pr[k] = (e < NS && star_node(g, fx, fy, e, nd)) ? r[(e / (S1 * S1)) * g.N + nd] : 0.f;
    }
  };
  fetch(item);
  for (;;) {
    int vx, vy;
    vertex(item, vx, vy);
    const long long v = (long long)vx + (long long)(g.n[0] + 1) * vy;
    __syncwarp();   // every lane has finished reading the previous star from ws / rs2
    float4* dst = reinterpret_cast<float4*>(&ws[w][0]);
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      const int e = lane + 32 * q;
      if (e < NV) dst[e] = pw[q];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int e = lane + 32 * k;
      if (e < NS) {
        rs2[w][e] = pr[k];
        rs2[w][e + NS] = pr[k];
      }
    }
    __syncwarp();
    const long long next = item + nwarps;
    if (next < count) fetch(next);   // in flight during this star's products
    // lane j < H owns rows j and j + H; row j takes step t while row j + H takes step
    // H - t, which reads the same two r values (r_(j+t) and r_(j-t mod NS)): six shared
    // reads per four FMAs instead of eight
    float acc[2] = {0.f, 0.f};
    const float* W = &ws[w][0];
    const float* rr = &rs2[w][0];
    if (lane < H) {
      const int j = lane;
#pragma unroll 2
      for (int t = 0; t <= H; ++t) {
        const float* wt = W + t * kWLD;         // W_t
        const float* wu = W + (H - t) * kWLD;   // W_(H-t)
        const float a = rr[j + t], b = rr[j - t + NS];
        acc[0] += wt[j] * a;
        if (t > 0 && t < H) {
          const int m = j - t < 0 ? j - t + NS : j - t;   // row m = j - t (mod NS) holds A(m, j)
          acc[0] += wt[m] * b;
          acc[1] += wu[j + t] * a;                        // A(j + t, j + H) r_(j+t)
        }
        acc[1] += wu[j + H] * b;                          // A(j + H, j - t) r_(j-t)
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (lane >= H) break;
      const int i = lane + H * k;
      if (!interior) {
        out[v * NS + i] = acc[k];
      } else {
        long long nd;
        if (star_node(g, vx, vy, i, nd)) {
          float* o = out + (i / (S1 * S1)) * g.N + nd;
          *o = mode == 2 ? *o - acc[k] : acc[k];
        }
      }
    }
    if (next >= count) break;
    item = next;
  }
}

// blocks of a k_qk_star_apply_w launch over `count` stars: one star a warp up to
// kStarWBlocksPerSM resident blocks an SM, beyond that the warps loop
static unsigned star_w_blocks(long long count) {
  static const int cap = [] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 152;
    }
    return kStarWBlocksPerSM * sms;
  }();
  const long long need = (count + 7) / 8;
  return (unsigned)(need < 1 ? 1 : need < cap ? need : cap);
}

// the wrapped FP32 rows from the FP64 packed diagonals (loading caller-supplied inverses)
__global__ void k_qk_wrap32(long long nverts, int pstride, const double* __restrict__ inv64,
                            float* __restrict__ inv32) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nverts * kWStride) return;
  const long long v = e / kWStride;
  const int rem = (int)(e % kWStride), t = rem / kWLD, i = rem % kWLD;
  float val = 0.f;
  if (i < NS) {
    const int j = i + t;
    const double* S = inv64 + v * pstride;
    val = (float)(j < NS ? S[diag_start(NS, t) + i] : S[diag_start(NS, NS - t) + (j - NS)]);
  }
  inv32[e] = val;
}

// z(node) = sum over the stars containing the node (vertices v with |i - 3v| <= 2 per
// axis), fixed order; 0 at Dirichlet nodes; divided by den[0] when den is given
template <typename T>
__global__ void k_qk_star_gather(Geom g, const T* __restrict__ sc, T* __restrict__ z, const T* __restrict__ den) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.N) return;
  const int comp = (int)(t / g.N);
  const long long nd = t - comp * g.N;
  const int i = (int)(nd % g.nn[0]), j = (int)(nd / g.nn[0]);
  if (i == 0 || i == g.nn[0] - 1 || j == 0 || j == g.nn[1] - 1) { z[t] = T(0); return; }
  int vxs[2], oxs[2], vys[2], oys[2], mx = 0, my = 0;
  { const int v0 = i / K, r = i - K * v0; vxs[mx] = v0; oxs[mx++] = r; if (r != 0) { vxs[mx] = v0 + 1; oxs[mx++] = r - K; } }
  { const int v0 = j / K, r = j - K * v0; vys[my] = v0; oys[my++] = r; if (r != 0) { vys[my] = v0 + 1; oys[my++] = r - K; } }
  T acc = T(0);
  for (int b = 0; b < my; ++b)
    for (int a = 0; a < mx; ++a) {
      const long long v = (long long)vxs[a] + (long long)(g.n[0] + 1) * vys[b];
      const int e = comp * S1 * S1 + (oxs[a] + K - 1) + S1 * (oys[b] + K - 1);
      acc += sc[v * NS + e];
    }
  if (den) acc = den[0] != T(0) ? acc / den[0] : T(0);
  z[t] = acc;
}

// ---------------------------------------------------------------------------
// transfers: P_H (coarse Q3 basis at the fine nodes, tensor product of 1D weights; each fine
// node belongs to the coarse cell min(f div 6, nc - 1)) and its transpose, as gathers;
// fine Dirichlet rows and coarse Dirichlet columns are zero
// ---------------------------------------------------------------------------
// coarse cell of fine lattice index f and its row of 1D weights
__device__ __forceinline__ int owner(int f, int nc, int& fr) {
  int c = f / (2 * K);
  if (c > nc - 1) c = nc - 1;
  fr = f - 2 * K * c;
  return c;
}

template <typename T>
__global__ void k_qk_prolong(Geom gc, Geom gf, const T* __restrict__ xc, T* __restrict__ xf, T* __restrict__ xadd) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * gf.N) return;
  const int comp = (int)(t / gf.N);
  const long long nd = t - comp * gf.N;
  const int i = (int)(nd % gf.nn[0]), j = (int)(nd / gf.nn[0]);
  T v = T(0);
  if (!(i == 0 || i == gf.nn[0] - 1 || j == 0 || j == gf.nn[1] - 1)) {
    int fx, fy;
    const int cx = owner(i, gc.n[0], fx), cy = owner(j, gc.n[1], fy);
    T acc = T(0);
    for (int b = 0; b < N1; ++b)
      for (int a = 0; a < N1; ++a) {
        const int I = K * cx + a, J = K * cy + b;
        if (I == 0 || I == gc.nn[0] - 1 || J == 0 || J == gc.nn[1] - 1) continue;
        acc += Tab<T>::pw(fx, a) * Tab<T>::pw(fy, b) * xc[comp * gc.N + I + (long long)gc.nn[0] * J];
      }
    v = acc;
  }
  xf[t] = v;
  if (xadd) xadd[t] += v;
}

// rc = P_H^T (rf - sub): coarse node J gathers the fine nodes owned by the coarse cells that
// contain it, weighted by its basis function there
template <typename T>
__global__ void k_qk_restrict(Geom gc, Geom gf, const T* __restrict__ rf, const T* __restrict__ sub, T* __restrict__ rc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * gc.N) return;
  const int comp = (int)(t / gc.N);
  const long long nd = t - comp * gc.N;
  const int I = (int)(nd % gc.nn[0]), J = (int)(nd / gc.nn[0]);
  if (I == 0 || I == gc.nn[0] - 1 || J == 0 || J == gc.nn[1] - 1) { rc[t] = T(0); return; }
  int cxs[2], axs[2], cys[2], ays[2];
  const int mx = cells_of(I, gc.n[0], cxs, axs), my = cells_of(J, gc.n[1], cys, ays);
  T acc = T(0);
  for (int b = 0; b < my; ++b)
    for (int a = 0; a < mx; ++a)
      for (int fy = 0; fy <= 2 * K; ++fy) {
        const int j = 2 * K * cys[b] + fy;
        if (fy == 2 * K && cys[b] != gc.n[1] - 1) continue;   // owned by the next coarse cell
        if (j == 0 || j == gf.nn[1] - 1) continue;
        const T wy = Tab<T>::pw(fy, ays[b]);
        if (wy == T(0)) continue;
        for (int fx = 0; fx <= 2 * K; ++fx) {
          const int i = 2 * K * cxs[a] + fx;
          if (fx == 2 * K && cxs[a] != gc.n[0] - 1) continue;
          if (i == 0 || i == gf.nn[0] - 1) continue;
          const T wx = Tab<T>::pw(fx, axs[a]);
          if (wx == T(0)) continue;
          const long long fn = comp * gf.N + i + (long long)gf.nn[0] * j;
          acc += wx * wy * (sub ? rf[fn] - sub[fn] : rf[fn]);
        }
      }
  rc[t] = acc;
}

}  // namespace qk

// ---------------------------------------------------------------------------
// entry points used by the dispatchers of operator.cu, patches.cu, transfer.cu, coarse.cu
// ---------------------------------------------------------------------------
void qk_tables() {
  qk::ensure_tables();
  qk3_tables();
}

void qk_apply(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y, const void* p_in, void* p_out,
              cudaStream_t s) {
  if (L.g.dim == 3) return qk3_apply(L, prec, mode, gamma, x, y, p_in, p_out, s);
  if (prec == PREC_F64) qk::apply_t<double>(L, mode, gamma, x, y, p_in, p_out, s);
  else qk::apply_t<float>(L, mode, gamma, x, y, p_in, p_out, s);
}

// op_apply_epi for order 3: the cell kernel of A_gamma (viscous + AL) into the staged
// outputs, then the gather with the Arnoldi epilogue
template <typename T>
static void apply_epi_t(const LevelDev& L, double gamma, const void* x, void* y, const ApplyEpi& e, cudaStream_t s,
                        cudaEvent_t e0, cudaEvent_t e1) {
  const T* mu = std::is_same<T, double>::value ? (const T*)L.coef64 : (const T*)L.coef32;
  const T* winv = std::is_same<T, double>::value ? (const T*)L.winv64 : (const T*)L.winv32;
  // External records become event-record nodes when the stream is being captured
  if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
  qk::k_qk_cells<T, OP_VISC | OP_AL><<<(unsigned)((L.g.ncells + 7) / 8), 256, 0, s>>>(
      L.g, qk::cell_scal<T>(L.g, gamma), (const T*)x, mu, winv, nullptr, nullptr, (T*)L.ebuf);
  if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
  qk::k_qk_gather_epi<T><<<(unsigned)((2 * L.g.N + RED_THREADS - 1) / RED_THREADS), RED_THREADS, 0, s>>>(
      L.g, (const T*)L.ebuf, (const T*)x, (T*)y, (const T*)e.b, e.sigma, e.k, (const T*)e.V, e.ld, (T*)e.out, e.start,
      e.st, e.partial);
  count_launch(2);
}

void qk_apply_epi(const LevelDev& L, int prec, double gamma, const void* x, void* y, const ApplyEpi& e,
                  cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  if (L.g.dim == 3) return qk3_apply_epi(L, prec, gamma, x, y, e, s, e0, e1);
  if (prec == PREC_F64) apply_epi_t<double>(L, gamma, x, y, e, s, e0, e1);
  else apply_epi_t<float>(L, gamma, x, y, e, s, e0, e1);
}

size_t qk_star32_floats(int dim) { return dim == 3 ? qk3_star32_floats() : (size_t)qk::kWStride; }

void qk_derive32(const LevelDev& L, cudaStream_t s) {
  if (L.g.dim == 3) return qk3_derive32(L, s);
  const long long tot = L.g.nverts * qk::kWStride;
  qk::k_qk_wrap32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.g.nverts, L.pstride, L.inv64, L.inv32);
  count_launch(1);
}

void qk_load_vector(const LevelDev& L, const double* f_qp, double* F, cudaStream_t s) {
  if (L.g.dim == 3) return qk3_load_vector(L, f_qp, F, s);
  const long long tot = L.g.ncells * qk::NE;
  qk::k_qk_load<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.g, f_qp, (double*)L.ebuf);
  qk::k_qk_gather<double><<<(unsigned)((2 * L.g.N + 255) / 256), 256, 0, s>>>(L.g, (const double*)L.ebuf, nullptr, F,
                                                                             0, 1);
  count_launch(2);
}

void qk_mass_setup(const LevelDev& L, double gamma, int w_mu, int variant, double* winv64, float* winv32, double* S,
                   DevStatus* st, cudaStream_t s) {
  if (L.g.dim == 3) return qk3_mass_setup(L, gamma, w_mu, variant, winv64, winv32, S, st, s);
  qk::k_qk_mass<<<(unsigned)((L.g.ncells + 127) / 128), 128, 0, s>>>(L.g, gamma, L.mu64, w_mu, variant, winv64, winv32,
                                                                     S, st);
  count_launch(1);
}

void qk_patch_setup(const LevelDev& L, double gamma, DevStatus* st, cudaStream_t s, int df64) {
  if (L.g.dim == 3) return qk3_patch_setup(L, gamma, st, s, df64);
  qk::k_qk_star_setup<<<(unsigned)L.g.nverts, 256, 0, s>>>(L.g, gamma, L.mu64, L.winv64, L.inv64, L.inv32, L.pstride,
                                                           st);
  count_launch(1);
}

void qk_patch_smooth(const LevelDev& L, int prec, const void* r, void* z, void* scratch, const void* den,
                     cudaStream_t s) {
  if (L.g.dim == 3) return qk3_patch_smooth(L, prec, r, z, scratch, den, s);
  const unsigned b2 = (unsigned)((2 * L.g.N + 255) / 256);
  constexpr int W64 = qk::star_warps<double>(), W32 = qk::star_warps<float>();
  if (prec == PREC_F64) {
    qk::k_qk_star_apply<double><<<(unsigned)((L.g.nverts + W64 - 1) / W64), 32 * W64, 0, s>>>(
        L.g, L.inv64, L.pstride, 0, 0, (const double*)r, (double*)scratch);
    qk::k_qk_star_gather<double><<<b2, 256, 0, s>>>(L.g, (const double*)scratch, (double*)z, (const double*)den);
  } else {
    qk::k_qk_star_apply_w<<<qk::star_w_blocks(L.g.nverts), 256, 0, s>>>(L.g, L.inv32, 0, 0, (const float*)r,
                                                                      (float*)scratch);
    qk::k_qk_star_gather<float><<<b2, 256, 0, s>>>(L.g, (const float*)scratch, (float*)z, (const float*)den);
  }
  count_launch(2);
}

void qk_interior_solve(const LevelDev& fine, int prec, const void* in, void* out, int subtract, cudaStream_t s) {
  if (fine.g.dim == 3) return qk3_interior_solve(fine, prec, in, out, subtract, s);
  const long long nc = (long long)(fine.g.n[0] / 2) * (fine.g.n[1] / 2);
  const size_t es = prec == PREC_F64 ? 8 : 4;
  if (!subtract) cudaMemsetAsync(out, 0, es * 2 * fine.g.N, s);
  constexpr int W64 = qk::star_warps<double>(), W32 = qk::star_warps<float>();
  if (prec == PREC_F64)
    qk::k_qk_star_apply<double><<<(unsigned)((nc + W64 - 1) / W64), 32 * W64, 0, s>>>(
        fine.g, fine.inv64, fine.pstride, 1, subtract ? 2 : 1, (const double*)in, (double*)out);
  else
    qk::k_qk_star_apply_w<<<qk::star_w_blocks(nc), 256, 0, s>>>(fine.g, fine.inv32, 1, subtract ? 2 : 1,
                                                              (const float*)in, (float*)out);
  count_launch(1);
}

void qk_prolong(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf, cudaStream_t s,
                void* xadd) {
  if (fine.g.dim == 3) return qk3_prolong(coarse, fine, prec, xc, xf, s, xadd);
  const unsigned b = (unsigned)((2 * fine.g.N + 255) / 256);
  if (prec == PREC_F64)
    qk::k_qk_prolong<double><<<b, 256, 0, s>>>(coarse.g, fine.g, (const double*)xc, (double*)xf, (double*)xadd);
  else qk::k_qk_prolong<float><<<b, 256, 0, s>>>(coarse.g, fine.g, (const float*)xc, (float*)xf, (float*)xadd);
  count_launch(1);
}

void qk_restrict(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc, cudaStream_t s,
                 const void* sub) {
  if (fine.g.dim == 3) return qk3_restrict(coarse, fine, prec, rf, rc, s, sub);
  const unsigned b = (unsigned)((2 * coarse.g.N + 255) / 256);
  if (prec == PREC_F64)
    qk::k_qk_restrict<double><<<b, 256, 0, s>>>(coarse.g, fine.g, (const double*)rf, (const double*)sub, (double*)rc);
  else qk::k_qk_restrict<float><<<b, 256, 0, s>>>(coarse.g, fine.g, (const float*)rf, (const float*)sub, (float*)rc);
  count_launch(1);
}

}  // namespace als
