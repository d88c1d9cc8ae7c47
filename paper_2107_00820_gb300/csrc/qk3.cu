// The order-3 discretisation in three dimensions: [Q3]^3 x P2^disc on uniform hexahedral
// meshes (the discretisation of the 3D sinker runs, Table linear, and the k = 3 column of
// Table k, Sec. 5.2.2), FP64 and FP32: operator applies, vertex-star setup and smoother,
// robust transfers, coarse images, mass and Schur blocks, so that the context's cycle and
// FGMRES run on it unchanged (qk.cu's entry points dispatch here for 3D levels).
//
// Velocity: continuous Q3, nodal basis on the 4 equispaced nodes -1, -1/3, 1/3, 1 per axis
// and cell, node lattice 3n + 1 per direction, x fastest; local node a = ax + 4 ay + 16 az.
// Pressure: discontinuous P2, the monomials in reference coordinates ordered by total
// degree, then x before y before z: {1, xi, eta, zeta, xi^2, xi eta, xi zeta, eta^2,
// eta zeta, zeta^2}; 10 per cell.  Quadrature: 4 x 4 x 4 Gauss-Legendre points, point
// q = qx + 4 qy + 16 qz.  Vertex stars: the free nodes at lattice offsets -2..2 from 3v in
// each direction (125 nodes, 375 dofs at an interior vertex); the interior of a coarse cell
// is the star of the fine vertex at its centre (Eq. (Ptilde)).
//
// The cell kernel factorises the tensor-product basis (sum factorisation: three 4-point
// contractions per direction instead of the 64 x 64 point-node products), one 64-thread
// group per cell.  The 375 x 375 star matrices do not fit in shared memory: each CTA of the
// persistent setup kernel assembles its star in a global workspace row block and inverts it
// by block Gauss-Jordan elimination (16 pivots per pass, the pivot block and the panels in
// shared memory).  Deterministic: per-cell and per-star outputs are staged and summed per
// node in a fixed order.
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "cell.cuh"
#include "df64.cuh"
#include "krylov.h"
#include "level.h"
#include "qk_tables.h"

namespace als {
namespace qk3 {

constexpr int K = 3;
constexpr int N1 = K + 1;          // nodes (and Gauss points) per axis and cell
constexpr int NB = N1 * N1 * N1;   // nodes per cell (64)
constexpr int NQ = NB;             // Gauss points per cell
constexpr int NPR = 10;            // pressure monomials per cell
constexpr int S1 = 2 * K - 1;      // star nodes per axis (5)
constexpr int SN = S1 * S1 * S1;   // star nodes (125)
constexpr int NS = 3 * SN;         // star dofs (375)
constexpr int NF = 2 * K + 1;      // fine lattice nodes per coarse cell and axis (7)
constexpr int CPB = 4;             // cells per block of the cell kernel (64 threads each)

__constant__ double cL[N1][N1], cD[N1][N1], cW[N1], cPSI[NQ][NPR], cPW[NF][N1];
// the FP32 cycle's copies (an FP64 operation costs ~70 FP32 ones here, conversions included)
// and the 3D point weights w_qx w_qy w_qz in both precisions
__constant__ float cLf[N1][N1], cDf[N1][N1], cPSIf[NQ][NPR], cPWf[NF][N1], cW3f[NQ];
__constant__ double cW3[NQ];
template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ double L(int q, int a) { return cL[q][a]; }
  static __device__ __forceinline__ double D(int q, int a) { return cD[q][a]; }
  static __device__ __forceinline__ double psi(int q, int p) { return cPSI[q][p]; }
  static __device__ __forceinline__ double pw(int f, int a) { return cPW[f][a]; }
  static __device__ __forceinline__ double w3(int q) { return cW3[q]; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ float L(int q, int a) { return cLf[q][a]; }
  static __device__ __forceinline__ float D(int q, int a) { return cDf[q][a]; }
  static __device__ __forceinline__ float psi(int q, int p) { return cPSIf[q][p]; }
  static __device__ __forceinline__ float pw(int f, int a) { return cPWf[f][a]; }
  static __device__ __forceinline__ float w3(int q) { return cW3f[q]; }
};
// per-level scalars of the cell kernel in its precision, formed on the host: the reference
// to physical derivative scales 2 / h_j, |J| = h0 h1 h2 / 8, and gamma
template <typename T>
struct CellScal {
  T s[3], wdet, gamma;
};
template <typename T>
static CellScal<T> cell_scal(const Geom& g, double gamma) {
  CellScal<T> c;
  for (int j = 0; j < 3; ++j) c.s[j] = (T)(2.0 / g.h[j]);
  c.wdet = (T)(0.125 * g.h[0] * g.h[1] * g.h[2]);
  c.gamma = (T)gamma;
  return c;
}

void ensure_tables() {
  static bool done = false;
  if (done) return;
  double G[N1], L[N1][N1], D[N1][N1], W[N1], PW[NF][N1], PSI[NQ][NPR];
  qk_tab::tables_1d(G, L, D, W, PW);
  const int ex[NPR][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                          {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
  for (int q = 0; q < NQ; ++q) {
    const double x[3] = {G[q % N1], G[(q / N1) % N1], G[q / (N1 * N1)]};
    for (int p = 0; p < NPR; ++p) PSI[q][p] = pow(x[0], ex[p][0]) * pow(x[1], ex[p][1]) * pow(x[2], ex[p][2]);
  }
  cudaMemcpyToSymbol(cL, L, sizeof(L));
  cudaMemcpyToSymbol(cD, D, sizeof(D));
  cudaMemcpyToSymbol(cW, W, sizeof(W));
  cudaMemcpyToSymbol(cPSI, PSI, sizeof(PSI));
  cudaMemcpyToSymbol(cPW, PW, sizeof(PW));
  float Lf[N1][N1], Df[N1][N1], PSIf[NQ][NPR], PWf[NF][N1], W3f[NQ];
  double W3[NQ];
  for (int q = 0; q < N1; ++q)
    for (int a = 0; a < N1; ++a) { Lf[q][a] = (float)L[q][a]; Df[q][a] = (float)D[q][a]; }
  for (int q = 0; q < NQ; ++q) {
    for (int p = 0; p < NPR; ++p) PSIf[q][p] = (float)PSI[q][p];
    W3[q] = W[q % N1] * W[(q / N1) % N1] * W[q / (N1 * N1)];
    W3f[q] = (float)W3[q];
  }
  for (int f = 0; f < NF; ++f)
    for (int a = 0; a < N1; ++a) PWf[f][a] = (float)PW[f][a];
  cudaMemcpyToSymbol(cLf, Lf, sizeof(Lf));
  cudaMemcpyToSymbol(cDf, Df, sizeof(Df));
  cudaMemcpyToSymbol(cPSIf, PSIf, sizeof(PSIf));
  cudaMemcpyToSymbol(cPWf, PWf, sizeof(PWf));
  cudaMemcpyToSymbol(cW3f, W3f, sizeof(W3f));
  cudaMemcpyToSymbol(cW3, W3, sizeof(W3));
  done = true;
}

__device__ __forceinline__ bool bnd_node(const Geom& g, int i, int j, int k) {
  return i == 0 || i == g.nn[0] - 1 || j == 0 || j == g.nn[1] - 1 || k == 0 || k == g.nn[2] - 1;
}
__device__ __forceinline__ double wq_of(int q, double wdet) {
  return cW[q % N1] * cW[(q / N1) % N1] * cW[q / (N1 * N1)] * wdet;
}

// ---------------------------------------------------------------------------
// operator apply: 64 threads per cell.  Forward: u at the 64 nodes -> the 3 x 3 velocity
// gradient at the 64 points by contractions along x, y, z; then the pressure moments
// (B u)_p = -sum_q w |J| psi_p div u (a 64-thread reduction), the AL field
// gamma psi . W^-1 B u and the flux s_cj = w |J| (2 mu eps_cj - P delta_cj) (2 / h_j);
// backward: y_c(a) = sum_q sum_j s_cj d_j phi_a by the transposed contractions z, y, x.
// ---------------------------------------------------------------------------
template <typename T>
struct CellShared {
  T L[N1][N1], D[N1][N1];
  T psi[NQ][NPR];
  T wq[NQ];
  T b0[CPB][9][NB];
  T b1[CPB][9][NB];
  T red[CPB][2][NPR];
  T sp[CPB][NPR];
};

template <typename T, int MODE>
__global__ void __launch_bounds__(64 * CPB) k_qk3_cells(Geom g, CellScal<T> cs, const T* __restrict__ x,
                                                        const T* __restrict__ mu, const T* __restrict__ winv,
                                                        const T* __restrict__ p_in, T* __restrict__ p_out,
                                                        T* __restrict__ ebuf) {
  constexpr bool RAW = (MODE & OP_RAW) != 0, VISC = (MODE & OP_VISC) != 0, AL = (MODE & OP_AL) != 0;
  constexpr bool BT = (MODE & OP_BT) != 0, BO = (MODE & OP_B) != 0;
  constexpr bool NEED_U = VISC || AL || BO, NEED_FLUX = VISC || AL || BT;
  __shared__ CellShared<T> sh;
  const int tid = threadIdx.x;
  if (tid < N1 * N1) {
    sh.L[tid / N1][tid % N1] = Tab<T>::L(tid / N1, tid % N1);
    sh.D[tid / N1][tid % N1] = Tab<T>::D(tid / N1, tid % N1);
  }
  for (int e = tid; e < NQ * NPR; e += blockDim.x) sh.psi[e / NPR][e % NPR] = Tab<T>::psi(e / NPR, e % NPR);
  if (tid < NQ) sh.wq[tid] = Tab<T>::w3(tid) * cs.wdet;
  const int w = tid >> 6, t = tid & 63, t0 = t & 3, t1 = (t >> 2) & 3, t2 = t >> 4;
  const long long cell = (long long)blockIdx.x * CPB + w;
  const bool valid = cell < g.ncells;
  const int cx = valid ? (int)(cell % g.n[0]) : 0;
  const int cy = valid ? (int)((cell / g.n[0]) % g.n[1]) : 0;
  const int cz = valid ? (int)(cell / ((long long)g.n[0] * g.n[1])) : 0;
  const T sx = cs.s[0], sy = cs.s[1], sz = cs.s[2];
  T(*b0)[NB] = sh.b0[w];
  T(*b1)[NB] = sh.b1[w];
  {
    const int i = K * cx + t0, j = K * cy + t1, k = K * cz + t2;
    const bool bnd = bnd_node(g, i, j, k);
    const long long nd = node_id(g, i, j, k);
    for (int c = 0; c < 3; ++c) b0[c][t] = (valid && NEED_U && (RAW || !bnd)) ? x[c * g.N + nd] : T(0);
  }
  __syncthreads();
  // x: (ax, ay, az) -> (qx, ay, az): A = L u, B = D u
  {
    const int qx = t0, base = N1 * t1 + N1 * N1 * t2;
    for (int c = 0; c < 3; ++c) {
      T a = T(0), b = T(0);
#pragma unroll
      for (int ax = 0; ax < N1; ++ax) {
        const T u = b0[c][base + ax];
        a += sh.L[qx][ax] * u;
        b += sh.D[qx][ax] * u;
      }
      b1[c][t] = a;
      b1[3 + c][t] = b;
    }
  }
  __syncthreads();
  // y: (qx, ay, az) -> (qx, qy, az): AL = L A, AD = D A, BL = L B
  {
    const int qy = t1, base = t0 + N1 * N1 * t2;
    for (int c = 0; c < 3; ++c) {
      T al = T(0), ad = T(0), bl = T(0);
#pragma unroll
      for (int ay = 0; ay < N1; ++ay) {
        const T a = b1[c][base + N1 * ay], b = b1[3 + c][base + N1 * ay];
        al += sh.L[qy][ay] * a;
        ad += sh.D[qy][ay] * a;
        bl += sh.L[qy][ay] * b;
      }
      b0[c][t] = al;
      b0[3 + c][t] = ad;
      b0[6 + c][t] = bl;
    }
  }
  __syncthreads();
  // z: (qx, qy, az) -> (qx, qy, qz): the gradient G[c][j] at point q = t
  T G[3][3];
  {
    const int qz = t2, base = t0 + N1 * t1;
    for (int c = 0; c < 3; ++c) {
      T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
      for (int az = 0; az < N1; ++az) {
        const int o = base + N1 * N1 * az;
        gx += sh.L[qz][az] * b0[6 + c][o];
        gy += sh.L[qz][az] * b0[3 + c][o];
        gz += sh.D[qz][az] * b0[c][o];
      }
      G[c][0] = gx * sx;
      G[c][1] = gy * sy;
      G[c][2] = gz * sz;
    }
  }
  const int q = t;
  const T div = G[0][0] + G[1][1] + G[2][2];
  T P = T(0);   // gamma pi + p_in at the point
  if (AL || BO) {
    // (B u)_p over the cell's 64 points: warp sums, then the two warps in a fixed order
    T bu[NPR];
#pragma unroll
    for (int p = 0; p < NPR; ++p) {
      T v = -sh.wq[q] * sh.psi[q][p] * div;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      bu[p] = v;
    }
    if ((t & 31) == 0)
      for (int p = 0; p < NPR; ++p) sh.red[w][t >> 5][p] = bu[p];
    __syncthreads();
    for (int p = 0; p < NPR; ++p) bu[p] = sh.red[w][0][p] + sh.red[w][1][p];
    if (BO && valid && t == 0)
      for (int p = 0; p < NPR; ++p) p_out[cell * NPR + p] = bu[p];
    if (AL) {
      if (valid && t < NPR) {
        const T* Wc = winv + cell * NPR * NPR;
        T s = T(0);
        for (int r = 0; r < NPR; ++r) s += Wc[t * NPR + r] * bu[r];
        sh.sp[w][t] = s;
      }
      __syncthreads();
      T pi = T(0);
      if (valid)
        for (int p = 0; p < NPR; ++p) pi += sh.psi[q][p] * sh.sp[w][p];
      P += cs.gamma * pi;
    }
  }
  if (BT && valid)
    for (int p = 0; p < NPR; ++p) P += sh.psi[q][p] * p_in[cell * NPR + p];
  if (!NEED_FLUX) return;   // uniform over the block
  {
    const T m2 = (VISC && valid) ? T(2) * mu[cell * NQ + q] : T(0);
    const T wq = sh.wq[q];
    const T sj[3] = {sx, sy, sz};
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < 3; ++j) {
        const T eps = T(0.5) * (G[c][j] + G[j][c]);
        b1[3 * c + j][t] = wq * (m2 * eps - (c == j ? P : T(0))) * sj[j];
      }
  }
  __syncthreads();
  // z^T: (qx, qy, qz) -> (qx, qy, az): T0 = L s_c0, T1 = L s_c1, T2 = D s_c2
  {
    const int az = t2, base = t0 + N1 * t1;
    for (int c = 0; c < 3; ++c) {
      T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
      for (int qz = 0; qz < N1; ++qz) {
        const int o = base + N1 * N1 * qz;
        s0 += sh.L[qz][az] * b1[3 * c][o];
        s1 += sh.L[qz][az] * b1[3 * c + 1][o];
        s2 += sh.D[qz][az] * b1[3 * c + 2][o];
      }
      b0[3 * c][t] = s0;
      b0[3 * c + 1][t] = s1;
      b0[3 * c + 2][t] = s2;
    }
  }
  __syncthreads();
  // y^T: (qx, qy, az) -> (qx, ay, az): V = L T0 (x derivative still to come), W = D T1 + L T2
  {
    const int ay = t1, base = t0 + N1 * N1 * t2;
    for (int c = 0; c < 3; ++c) {
      T v = T(0), wv = T(0);
#pragma unroll
      for (int qy = 0; qy < N1; ++qy) {
        const int o = base + N1 * qy;
        v += sh.L[qy][ay] * b0[3 * c][o];
        wv += sh.D[qy][ay] * b0[3 * c + 1][o] + sh.L[qy][ay] * b0[3 * c + 2][o];
      }
      b1[c][t] = v;
      b1[3 + c][t] = wv;
    }
  }
  __syncthreads();
  // x^T: (qx, ay, az) -> (ax, ay, az): y_c = D V + L W
  if (valid) {
    const int ax = t0, base = N1 * t1 + N1 * N1 * t2;
    for (int c = 0; c < 3; ++c) {
      T y = T(0);
#pragma unroll
      for (int qx = 0; qx < N1; ++qx) y += sh.D[qx][ax] * b1[c][base + qx] + sh.L[qx][ax] * b1[3 + c][base + qx];
      ebuf[(cell * 3 + c) * NB + t] = y;
    }
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

// y(node) = sum of the staged cell outputs of the (up to 8) cells containing it, fixed
// order; keep_bnd: y = x at Dirichlet nodes; raw: no Dirichlet treatment
template <typename T>
__device__ __forceinline__ T gather_value(const Geom& g, const T* __restrict__ ebuf, const T* __restrict__ x,
                                          long long t, int keep_bnd, int raw) {
  const int comp = (int)(t / g.N);
  const long long nd = t - comp * g.N;
  const int i = (int)(nd % g.nn[0]);
  const long long r = nd / g.nn[0];
  const int j = (int)(r % g.nn[1]), k = (int)(r / g.nn[1]);
  if (bnd_node(g, i, j, k) && !raw) return keep_bnd ? x[t] : T(0);
  int cxs[2], axs[2], cys[2], ays[2], czs[2], azs[2];
  const int mx = cells_of(i, g.n[0], cxs, axs), my = cells_of(j, g.n[1], cys, ays), mz = cells_of(k, g.n[2], czs, azs);
  T acc = T(0);
  for (int c = 0; c < mz; ++c)
    for (int b = 0; b < my; ++b)
      for (int a = 0; a < mx; ++a) {
        const long long cell = (long long)cxs[a] + (long long)g.n[0] * ((long long)cys[b] + (long long)g.n[1] * czs[c]);
        acc += ebuf[(cell * 3 + comp) * NB + axs[a] + N1 * ays[b] + N1 * N1 * azs[c]];
      }
  return acc;
}

template <typename T>
__global__ void k_qk3_gather(Geom g, const T* __restrict__ ebuf, const T* __restrict__ x, T* __restrict__ y,
                             int keep_bnd, int raw) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * g.N) return;
  y[t] = gather_value<T>(g, ebuf, x, t, keep_bnd, raw);
}

// the gather fused with the GMRES smoother's Arnoldi reduction (as for the other
// discretisations): y = b + sigma A x; start = 0: out[j] = (V_j . y) / hn[j], j < k;
// start = 1: |y|^2 starts the GMRES cycle.  Block partials in a fixed order.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_qk3_gather_epi(Geom g, const T* __restrict__ ebuf,
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
  if (t < 3 * g.N) {
    const T v = (b ? b[t] : T(0)) + (T)sigma * gather_value<T>(g, ebuf, x, t, 1, 0);
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
  k_qk3_cells<T, MODE><<<(unsigned)((L.g.ncells + CPB - 1) / CPB), 64 * CPB, 0, s>>>(
      L.g, cell_scal<T>(L.g, gamma), (const T*)x, mu, winv, (const T*)p_in, (T*)p_out, (T*)L.ebuf);
  if (NEED_FLUX) {
    const int keep = ((MODE & OP_VISC) && !(MODE & OP_RAW)) ? 1 : 0;
    k_qk3_gather<T><<<(unsigned)((3 * L.g.N + 255) / 256), 256, 0, s>>>(L.g, (const T*)L.ebuf, (const T*)x, (T*)y,
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

template <typename T>
static void apply_epi_t(const LevelDev& L, double gamma, const void* x, void* y, const ApplyEpi& e, cudaStream_t s,
                        cudaEvent_t e0, cudaEvent_t e1) {
  const T* mu = std::is_same<T, double>::value ? (const T*)L.coef64 : (const T*)L.coef32;
  const T* winv = std::is_same<T, double>::value ? (const T*)L.winv64 : (const T*)L.winv32;
  // External records become event-record nodes when the stream is being captured
  if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
  k_qk3_cells<T, OP_VISC | OP_AL><<<(unsigned)((L.g.ncells + CPB - 1) / CPB), 64 * CPB, 0, s>>>(
      L.g, cell_scal<T>(L.g, gamma), (const T*)x, mu, winv, nullptr, nullptr, (T*)L.ebuf);
  if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
  k_qk3_gather_epi<T><<<(unsigned)((3 * L.g.N + RED_THREADS - 1) / RED_THREADS), RED_THREADS, 0, s>>>(
      L.g, (const T*)L.ebuf, (const T*)x, (T*)y, (const T*)e.b, e.sigma, e.k, (const T*)e.V, e.ld, (T*)e.out, e.start,
      e.st, e.partial);
  count_launch(2);
}

// F_(c,a) = sum_q |J| w_q f_c(x_q) phi_a(x_q), staged per cell, summed per node; f is
// [cell][q][3]
__global__ void k_qk3_load(Geom g, const double* __restrict__ f, double* __restrict__ ebuf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ncells * 3 * NB) return;
  const long long cell = t / (3 * NB);
  const int e = (int)(t % (3 * NB)), comp = e / NB, a = e % NB;
  const int ax = a % N1, ay = (a / N1) % N1, az = a / (N1 * N1);
  const double wdet = 0.125 * g.h[0] * g.h[1] * g.h[2];
  double acc = 0.0;
  for (int q = 0; q < NQ; ++q) {
    const double phi = cL[q % N1][ax] * cL[(q / N1) % N1][ay] * cL[q / (N1 * N1)][az];
    acc += wq_of(q, wdet) * f[(cell * NQ + q) * 3 + comp] * phi;
  }
  ebuf[(cell * 3 + comp) * NB + a] = acc;
}

// ---------------------------------------------------------------------------
// per-cell mass blocks: M_K(1/mu)^-1 and M_K^-1 (10 x 10, Gauss-Jordan), the augmentation
// weight's inverse W^-1 (W = M_p or M_p(1/mu)) and the Schur blocks S of Eq. (P1P2):
// P1: M_K(1/mu)^-1 + gamma M_K^-1, P2: (1 + gamma) M_K(1/mu)^-1.  One thread per cell.
// ---------------------------------------------------------------------------
__device__ void inv10(double (&A)[NPR][NPR], DevStatus* st, long long where) {
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

__global__ void k_qk3_mass(Geom g, double gamma, const double* __restrict__ mu, int w_mu, int variant,
                           double* __restrict__ winv64, float* __restrict__ winv32, double* __restrict__ S,
                           DevStatus* st) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= g.ncells) return;
  const double wdet = 0.125 * g.h[0] * g.h[1] * g.h[2];
  double Mm[NPR][NPR], M[NPR][NPR];
  for (int p = 0; p < NPR; ++p)
    for (int r = 0; r < NPR; ++r) { Mm[p][r] = 0.0; M[p][r] = 0.0; }
  for (int q = 0; q < NQ; ++q) {
    const double wq = wq_of(q, wdet);
    const double im = 1.0 / mu[cell * NQ + q];
    for (int p = 0; p < NPR; ++p)
      for (int r = 0; r < NPR; ++r) {
        M[p][r] += wq * cPSI[q][p] * cPSI[q][r];
        Mm[p][r] += wq * im * cPSI[q][p] * cPSI[q][r];
      }
  }
  inv10(Mm, st, cell);
  inv10(M, st, cell);
  for (int p = 0; p < NPR; ++p)
    for (int r = 0; r < NPR; ++r) {
      const double wv = w_mu ? Mm[p][r] : M[p][r];
      if (winv64) winv64[cell * NPR * NPR + p * NPR + r] = wv;
      if (winv32) winv32[cell * NPR * NPR + p * NPR + r] = (float)wv;
      if (S) S[cell * NPR * NPR + p * NPR + r] = variant == 0 ? Mm[p][r] + gamma * M[p][r] : (1.0 + gamma) * Mm[p][r];
    }
}

// ---------------------------------------------------------------------------
// vertex stars: setup (assembly from the star's 8 cells into a workspace row block in
// global memory, block Gauss-Jordan inversion, FP64 packed-by-diagonals and its FP32
// rounding), products, node gather
// ---------------------------------------------------------------------------
// star entry e = comp * 125 + (ox + 2) + 5 (oy + 2) + 25 (oz + 2) of vertex v: node 3v + o
__device__ __forceinline__ bool star_node(const Geom& g, int vx, int vy, int vz, int e, long long& nd) {
  const int o = e % SN;
  const int i = K * vx + o % S1 - (K - 1), j = K * vy + (o / S1) % S1 - (K - 1), k = K * vz + o / (S1 * S1) - (K - 1);
  if (i <= 0 || i >= g.nn[0] - 1 || j <= 0 || j >= g.nn[1] - 1 || k <= 0 || k >= g.nn[2] - 1) return false;
  nd = node_id(g, i, j, k);
  return true;
}

constexpr int LDM = NS + 1;   // row stride of a star matrix in the workspace (doubles)
// FP32 star storage in wrapped rows (k_qk3_star_apply_w): WT rows of WLD entries
constexpr int WT = (NS + 1) / 2;   // 188
constexpr int WLD = 376;
constexpr int WSTRIDE = WT * WLD;
static_assert(NS % 2 == 1 && WLD % 4 == 0 && WLD >= NS, "wrapped-row layout");
static_assert(WT % 2 == 0, "rows are streamed in pairs");
constexpr int BB = 16;        // pivots per Gauss-Jordan pass
constexpr int SETUP_THREADS = 256;
// shared memory of the setup kernel (doubles): the assembly's tables or the elimination's
// pivot block and panels, whichever is larger
constexpr int ASM_DOUBLES = NQ * 27 * 3 + NQ + 2 * NPR * 81 + 8 * 3 * 3;
constexpr int GJ_DOUBLES = BB * BB + 2 * BB * NS + 2 * BB;
constexpr int SETUP_DOUBLES = ASM_DOUBLES > GJ_DOUBLES ? ASM_DOUBLES : GJ_DOUBLES;
constexpr size_t SETUP_SMEM = sizeof(double) * SETUP_DOUBLES + 16;

// entry e (0 <= e < N (N + 1) / 2) of the upper triangle of an N x N matrix, N odd, as
// (i, j), i <= j: the rows are taken in pairs (p, N - 1 - p), p < (N - 1) / 2, of N + 1
// entries together, then the middle row (consecutive e: consecutive j)
template <int N>
__device__ __forceinline__ void tri_entry(int e, int& i, int& j) {
  static_assert(N % 2 == 1, "odd order");
  constexpr int HALF = (N - 1) / 2;
  const int p = e / (N + 1), off = e - p * (N + 1);
  if (p < HALF) {
    if (off < N - p) { i = p; j = p + off; }
    else { i = N - 1 - p; j = i + off - (N - p); }
  } else {
    i = HALF;
    j = HALF + off;
  }
}

// One CTA per star at a time (persistent over the stars v = blockIdx.x, += gridDim.x), its
// star matrix in ws + blockIdx.x * NS * LDM.
// RM: the arithmetic of the elimination, double or DF64 (double-float, about 48 bits, on
// the FP32 pipes; the assembly is FP64 either way)
template <typename RM>
__global__ void __launch_bounds__(SETUP_THREADS) k_qk3_star_setup(Geom g, double gamma, const double* __restrict__ mu,
                                                                  const double* __restrict__ winv,
                                                                  double* __restrict__ ws, double* __restrict__ inv64,
                                                                  float* __restrict__ inv32, int pstride,
                                                                  DevStatus* st) {
  static_assert(sizeof(RM) == sizeof(double), "the workspace holds 8-byte entries");
  using Ops = RealOps<RM>;
  extern __shared__ double smem[];
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* M = ws + (long long)blockIdx.x * NS * LDM;
  const double sx = 2.0 / g.h[0], sy = 2.0 / g.h[1], sz = 2.0 / g.h[2];
  const double wdet = 0.125 * g.h[0] * g.h[1] * g.h[2];
  for (long long v = blockIdx.x; v < g.nverts; v += gridDim.x) {
    const int vx = (int)(v % g.nv[0]), vy = (int)((v / g.nv[0]) % g.nv[1]), vz = (int)(v / ((long long)g.nv[0] * g.nv[1]));
    if (tid == 0) s_bad = 0;
    for (int e = tid; e < NS * LDM; e += nt) M[e] = 0.0;
    __syncthreads();
    // ---- assembly: the cells (cx, cy, cz) in {v-1, v}^3 inside the mesh
    double* gq = smem;                      // [q][n][3]: d_j phi_n at q, the cell's 27 star nodes n
    double* wm = gq + NQ * 27 * 3;          // [q]: w |J| mu
    double* Bm = wm + NQ;                   // [p][c * 27 + n]: -sum_q w |J| psi_p d_c phi_n
    double* WB = Bm + NPR * 81;             // W^-1 Bm
    for (int cc = 0; cc < 8; ++cc) {
      const int cx = vx - 1 + (cc & 1), cy = vy - 1 + ((cc >> 1) & 1), cz = vz - 1 + (cc >> 2);
      if (cx < 0 || cy < 0 || cz < 0 || cx >= g.n[0] || cy >= g.n[1] || cz >= g.n[2]) continue;   // uniform
      const long long cell = (long long)cx + (long long)g.n[0] * ((long long)cy + (long long)g.n[1] * cz);
      // the star's nodes in this cell: local index a = m + off per axis, m = 0..2
      const int offx = cx == vx - 1 ? 1 : 0, offy = cy == vy - 1 ? 1 : 0, offz = cz == vz - 1 ? 1 : 0;
      for (int e = tid; e < NQ * 27; e += nt) {
        const int q = e / 27, n = e % 27;
        const int ax = n % 3 + offx, ay = (n / 3) % 3 + offy, az = n / 9 + offz;
        const int qx = q % N1, qy = (q / N1) % N1, qz = q / (N1 * N1);
        gq[e * 3 + 0] = cD[qx][ax] * cL[qy][ay] * cL[qz][az] * sx;
        gq[e * 3 + 1] = cL[qx][ax] * cD[qy][ay] * cL[qz][az] * sy;
        gq[e * 3 + 2] = cL[qx][ax] * cL[qy][ay] * cD[qz][az] * sz;
      }
      for (int q = tid; q < NQ; q += nt) wm[q] = wq_of(q, wdet) * mu[cell * NQ + q];
      __syncthreads();
      for (int e = tid; e < NPR * 81; e += nt) {
        const int p = e / 81, j = e % 81, c = j / 27, n = j % 27;
        double acc = 0.0;
        for (int q = 0; q < NQ; ++q) acc -= wq_of(q, wdet) * cPSI[q][p] * gq[(q * 27 + n) * 3 + c];
        Bm[e] = acc;
      }
      __syncthreads();
      const double* Wc = winv + cell * NPR * NPR;
      for (int e = tid; e < NPR * 81; e += nt) {
        const int p = e / 81, j = e % 81;
        double acc = 0.0;
        for (int r = 0; r < NPR; ++r) acc += Wc[p * NPR + r] * Bm[r * 81 + j];
        WB[e] = acc;
      }
      __syncthreads();
      // node pairs: H[a][b] = sum_q w |J| mu d_a phi_ni d_b phi_nj; the element entry of
      // (ci, ni), (cj, nj) is 2 mu eps(phi_ni e_ci) : eps(phi_nj e_cj) integrated,
      // = delta_(ci cj) trace H + H[cj][ci], plus gamma (B^T W^-1 B)
      for (int e = tid; e < 27 * 28 / 2; e += nt) {   // unordered node pairs ni <= nj
        int ni, nj;
        tri_entry<27>(e, ni, nj);
        double H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int q = 0; q < NQ; ++q) {
          const double* gi = gq + (q * 27 + ni) * 3;
          const double* gj = gq + (q * 27 + nj) * 3;
          const double wv = wm[q];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const double wa = wv * gi[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) H[a][b] += wa * gj[b];
          }
        }
        const double tr = H[0][0] + H[1][1] + H[2][2];
        const int sni = (ni % 3 + offx + K * cx - K * vx + 2) + S1 * ((ni / 3) % 3 + offy + K * cy - K * vy + 2) +
                        S1 * S1 * (ni / 9 + offz + K * cz - K * vz + 2);
        const int snj = (nj % 3 + offx + K * cx - K * vx + 2) + S1 * ((nj / 3) % 3 + offy + K * cy - K * vy + 2) +
                        S1 * S1 * (nj / 9 + offz + K * cz - K * vz + 2);
        // the 9 entries of the node block (ni, nj), each into the upper triangle (the
        // block (nj, ni) holds their transposes; for ni == nj only ci <= cj)
        for (int ci = 0; ci < 3; ++ci)
          for (int cj = 0; cj < 3; ++cj) {
            if (ni == nj && ci > cj) continue;
            double al = 0.0;
            for (int p = 0; p < NPR; ++p) al += Bm[p * 81 + ci * 27 + ni] * WB[p * 81 + cj * 27 + nj];
            const int si = ci * SN + sni, sj = cj * SN + snj;
            const int lo = si < sj ? si : sj, hi = si < sj ? sj : si;
            M[(long long)lo * LDM + hi] += (ci == cj ? tr : 0.0) + H[cj][ci] + gamma * al;
          }
      }
      __syncthreads();
    }
    // identity rows and columns at absent and Dirichlet nodes; the entries in the
    // elimination's arithmetic RM from here on (each thread converts its own entries).
    // From here only the upper triangle i <= j is kept (see the elimination below).
    RM* Mr = reinterpret_cast<RM*>(M);
    for (int e = tid; e < NS * (NS + 1) / 2; e += nt) {
      int i, j;
      tri_entry<NS>(e, i, j);
      long long nd;
      const bool fi = star_node(g, vx, vy, vz, i, nd), fj = star_node(g, vx, vy, vz, j, nd);
      const double val = (!fi || !fj) ? (i == j ? 1.0 : 0.0) : M[(long long)i * LDM + j];
      Mr[(long long)i * LDM + j] = Ops::from(val);
    }
    __syncthreads();
    // ---- block Gauss-Jordan inversion in place on the upper triangle (SPD: the pivot
    // blocks are Schur complements, no pivoting).  Per pass over pivots K = [k0, k0 + b):
    // Dk = M_KK^-1, C = M_.K (column panel), R = Dk M_K. (row panel); then M_KK = Dk,
    // M_Kj = R_j, M_iK = -C_i Dk, M_ij -= C_i R_j.  With s_x = -1 for the indices swept
    // so far and +1 for the others, every pass keeps M_ji = s_i s_j M_ij, so the upper
    // triangle determines the rest: X_x = M(min(x, K), max(x, K)) is C_x, and the raw row
    // panel is sigma_x X_x (sigma_x = -1 for x < k0, +1 beyond K).  With Y_x = Dk X_x the
    // pass sets M_ij -= sigma_j X_i . Y_j (i <= j outside K), M_iK = -Y_i (i < k0),
    // M_Kj = Y_j (j beyond K), M_KK = Dk; at the end all signs agree and M is A^-1.
    RM* Dk = reinterpret_cast<RM*>(smem);   // [BB][BB]
    RM* Yp = Dk + BB * BB;                  // [BB][NS]
    RM* C = Yp + BB * NS;                   // [NS][BB]: X
    RM* rowk = C + NS * BB;                 // [BB]
    RM* colk = rowk + BB;                   // [BB]
    const RM zero = Ops::from(0.0), one = Ops::from(1.0);
    for (int k0 = 0; k0 < NS; k0 += BB) {
      const int b = NS - k0 < BB ? NS - k0 : BB;
      for (int e = tid; e < BB * BB; e += nt) {
        const int m = e / BB, l = e % BB, lo = m < l ? m : l, hi = m < l ? l : m;
        Dk[e] = (m < b && l < b) ? Mr[(long long)(k0 + lo) * LDM + k0 + hi] : (m == l ? one : zero);
      }
      for (int e = tid; e < NS * BB; e += nt) {
        const int x = e / BB, l = e % BB, k = k0 + l;
        const bool inK = x >= k0 && x < k0 + b;
        C[e] = (l < b && !inK) ? (x < k ? Mr[(long long)x * LDM + k] : Mr[(long long)k * LDM + x]) : zero;
      }
      __syncthreads();
      for (int kk = 0; kk < b; ++kk) {   // scalar Gauss-Jordan on the pivot block
        const RM pv = Dk[kk * BB + kk];
        const bool ok = pv > 0.0f;
        if (!ok && tid == 0 && !s_bad) { report(st, 4 /* ALS_ENOTSPD */, v); s_bad = 1; }
        const RM ip = ok ? one / pv : one;
        if (tid < BB) {
          rowk[tid] = Dk[kk * BB + tid] * ip;
          colk[tid] = Dk[tid * BB + kk];
        }
        __syncthreads();
        if (tid < BB * BB) {
          const int m = tid / BB, l = tid % BB;
          RM val;
          if (m == kk && l == kk) val = ip;
          else if (m == kk) val = rowk[l];
          else if (l == kk) val = -(colk[m] * ip);
          else val = Ops::sub_prod(Dk[tid], colk[m], rowk[l]);
          Dk[tid] = val;
        }
        __syncthreads();
      }
      for (int e = tid; e < BB * NS; e += nt) {
        const int m = e / NS, x = e % NS;
        RM acc = zero;
        if (m < b)
          for (int l = 0; l < b; ++l) acc = Ops::add_prod(acc, Dk[m * BB + l], C[x * BB + l]);
        Yp[e] = acc;
      }
      __syncthreads();
      // EPT entries per thread at a time, EPT independent chains: the chain of one entry
      // is a sequence of dependent operations (16 double-float updates of ~15 FP32
      // instructions each), so the entries of a thread interleave to hide its latency
      constexpr int EPT = 4;
      constexpr int NT = NS * (NS + 1) / 2;
      for (int e0 = tid; e0 < NT; e0 += EPT * nt) {
        RM acc[EPT];
        const RM* xi[EPT];
        int jj[EPT];
        bool neg[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int e = e0 + q * nt;
          int i, j;
          tri_entry<NS>(e < NT ? e : 0, i, j);
          xi[q] = C + i * BB;
          jj[q] = j;
          neg[q] = j < k0;   // sigma_j = -1: the chain runs on -M_ij and is negated back
          const RM m = Mr[(long long)i * LDM + j];
          acc[q] = neg[q] ? -m : m;
        }
#pragma unroll
        for (int l = 0; l < BB; ++l)
#pragma unroll
          for (int q = 0; q < EPT; ++q) acc[q] = Ops::sub_prod(acc[q], xi[q][l], Yp[l * NS + jj[q]]);
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int e = e0 + q * nt;
          if (e >= NT) continue;
          int i, j;
          tri_entry<NS>(e, i, j);
          const int mi = i - k0, mj = j - k0;
          const bool ik = mi >= 0 && mi < b, jk = mj >= 0 && mj < b;
          RM val = neg[q] ? -acc[q] : acc[q];
          if (ik && jk) val = Dk[mi * BB + mj];
          else if (jk) val = -Yp[mj * NS + i];
          else if (ik) val = Yp[mi * NS + j];
          Mr[(long long)i * LDM + j] = val;
        }
      }
      __syncthreads();
    }
    // FP64: upper triangle by diagonals (entry (i, i + t)); FP32: the wrapped rows
    for (int t = 0; t < NS; ++t) {
      const long long base = v * pstride + diag_start(NS, t);
      for (int i = tid; i + t < NS; i += nt) inv64[base + i] = Ops::to_double(Mr[(long long)i * LDM + i + t]);
    }
    for (int e = tid; e < WSTRIDE; e += nt) {
      const int t = e / WLD, i = e % WLD, j = i + t < NS ? i + t : i + t - NS;
      const int lo = i < j ? i : j, hi = i < j ? j : i;
      inv32[v * WSTRIDE + e] = i < NS ? (float)Ops::to_double(Mr[(long long)lo * LDM + hi]) : 0.f;
    }
    __syncthreads();
  }
}


// y_v = A_v^-1 r|_v: one CTA of STAR_THREADS per star (vertex), rows by threads, over the
// wrapped diagonals (row i takes entry (i, (i + t) mod NS) at step t: entry i of diagonal t
// while i + t < NS, else entry i + t - NS of diagonal NS - t, its symmetric partner), so
// every thread multiplies at every step and each diagonal is read by consecutive threads.
// interior: the stars of the fine vertices 2c + 1 at the coarse-cell centres, written
// (mode 1) or subtracted (mode 2) straight into the nodes; else into the rows [vertex][375].
constexpr int STAR_THREADS = 128;
constexpr int STAR_ROWS = (NS + STAR_THREADS - 1) / STAR_THREADS;

template <typename T>
__global__ void __launch_bounds__(STAR_THREADS) k_qk3_star_apply(Geom g, const T* __restrict__ inv, int pstride,
                                                                 int interior, int mode, const T* __restrict__ r,
                                                                 T* __restrict__ out) {
  __shared__ T rs[NS];
  const int tid = threadIdx.x;
  const int ic[3] = {g.n[0] / 2, g.n[1] / 2, g.n[2] / 2};
  const long long count = interior ? (long long)ic[0] * ic[1] * ic[2] : g.nverts;
  const long long item = blockIdx.x;
  if (item >= count) return;   // uniform over the block
  int vx, vy, vz;
  if (interior) {
    vx = 2 * (int)(item % ic[0]) + 1;
    vy = 2 * (int)((item / ic[0]) % ic[1]) + 1;
    vz = 2 * (int)(item / ((long long)ic[0] * ic[1])) + 1;
  } else {
    vx = (int)(item % g.nv[0]);
    vy = (int)((item / g.nv[0]) % g.nv[1]);
    vz = (int)(item / ((long long)g.nv[0] * g.nv[1]));
  }
  const long long v = (long long)vx + (long long)g.nv[0] * ((long long)vy + (long long)g.nv[1] * vz);
  for (int e = tid; e < NS; e += STAR_THREADS) {
    long long nd;
    rs[e] = star_node(g, vx, vy, vz, e, nd) ? r[(e / SN) * g.N + nd] : T(0);
  }
  __syncthreads();
  const T* S = inv + v * pstride;
  T acc[STAR_ROWS];
#pragma unroll
  for (int k = 0; k < STAR_ROWS; ++k) acc[k] = T(0);
  // steps t and NS - t in the same iteration (NS is odd): both read the same two diagonals
  // (t and NS - t), each entry once for its row and once for its symmetric partner's, so
  // the second read of an entry follows the first within the iteration and hits in L1
  // instead of coming back from HBM
#pragma unroll
  for (int k = 0; k < STAR_ROWS; ++k) {
    const int i = tid + STAR_THREADS * k;
    if (i < NS) acc[k] += __ldg(S + i) * rs[i];   // t = 0: the main diagonal
  }
#pragma unroll 2
  for (int t = 1; t <= NS / 2; ++t) {
    const int u = NS - t;
    const T* dt = S + diag_start(NS, t);   // diagonal t (NS - t entries)
    const T* du = S + diag_start(NS, u);   // diagonal NS - t (t entries)
#pragma unroll
    for (int k = 0; k < STAR_ROWS; ++k) {
      const int i = tid + STAR_THREADS * k;
      if (i < NS) {
        // step t: entry (i, i + t) on diagonal t, else (i + t - NS, i) on diagonal NS - t;
        // step NS - t: entry (i, i + NS - t) on diagonal NS - t, else (i - t, i) on diagonal t
        const bool a = i < u, b = i < t;
        const T* p1 = a ? dt + i : du + (i - u);   // one load each, from the selected diagonal
        const T* p2 = b ? du + i : dt + (i - t);
        acc[k] += __ldg(p1) * rs[a ? i + t : i - u];
        acc[k] += __ldg(p2) * rs[b ? i + u : i - t];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < STAR_ROWS; ++k) {
    const int i = tid + STAR_THREADS * k;
    if (i >= NS) continue;
    if (!interior) {
      out[v * NS + i] = acc[k];
    } else {
      long long nd;
      if (star_node(g, vx, vy, vz, i, nd)) {
        T* o = out + (i / SN) * g.N + nd;
        *o = mode == 2 ? *o - acc[k] : acc[k];
      }
    }
  }
}

// FP32 star storage, "wrapped rows": for odd NS every unordered pair {i, j}, i != j, has a
// circular distance t = (j - i) mod NS or NS - t in 1..(NS - 1) / 2, so the symmetric
// matrix is the WT = (NS + 1) / 2 rows W_t[i] = A(i, (i + t) mod NS), t = 0..WT - 1, each
// padded to WLD = 376 entries (16-byte rows) -- 70,688 floats per star against 70,500 for
// the packed triangle.  The product y_i = sum_t W_t[i] r_(i+t) + sum_(t>0) W_t[i-t] r_(i-t)
// (indices mod NS) then reads each row once, coalesced, 16 bytes a thread.

// y_v = A_v^-1 r|_v from the wrapped rows: one CTA per star, rows by threads; the rows of
// W stream through shared memory two at a time (double-buffered, the next pair's 16-byte
// loads in flight while the current pair is used); r is held twice over so that
// r_((i + t) mod NS) needs no wrap.  interior / mode as k_qk3_star_apply.
constexpr int WV = WLD / 4;   // float4 per row (94)
// The rows' storage: FP32, or bfloat16 (ALS_STORE_BF16: the same rows rounded to nearest
// from FP64, 752-byte rows), widened to FP32 on the way into shared memory; every product
// and sum in FP32 either way.  A pair of rows is 188 16-byte words in FP32 (thread tid
// loads words tid and tid + 128) and 94 in bfloat16 (8 entries a word, threads 0..93).
template <typename TS>
struct RowPair;
template <>
struct RowPair<float> {
  float4 a, b;
  __device__ __forceinline__ void load(const float* base, int tid) {
    const float4* W = reinterpret_cast<const float4*>(base);
    a = __ldg(W + tid);
    b = tid + STAR_THREADS < 2 * WV ? __ldg(W + tid + STAR_THREADS) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __device__ __forceinline__ void store(float* w, int tid) const {
    reinterpret_cast<float4*>(w)[tid] = a;
    if (tid + STAR_THREADS < 2 * WV) reinterpret_cast<float4*>(w)[tid + STAR_THREADS] = b;
  }
};
template <>
struct RowPair<__nv_bfloat16> {
  uint4 a;
  __device__ __forceinline__ void load(const __nv_bfloat16* base, int tid) {
    a = tid < WV ? __ldg(reinterpret_cast<const uint4*>(base) + tid) : make_uint4(0u, 0u, 0u, 0u);
  }
  __device__ __forceinline__ void store(float* w, int tid) const {
    if (tid >= WV) return;
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&a);
    const float2 p0 = __bfloat1622float2(h[0]), p1 = __bfloat1622float2(h[1]);
    const float2 p2 = __bfloat1622float2(h[2]), p3 = __bfloat1622float2(h[3]);
    reinterpret_cast<float4*>(w)[2 * tid] = make_float4(p0.x, p0.y, p1.x, p1.y);
    reinterpret_cast<float4*>(w)[2 * tid + 1] = make_float4(p2.x, p2.y, p3.x, p3.y);
  }
};

template <typename TS>
__global__ void __launch_bounds__(STAR_THREADS) k_qk3_star_apply_w(Geom g, const TS* __restrict__ inv,
                                                                   int interior, int mode,
                                                                   const float* __restrict__ r,
                                                                   float* __restrict__ out) {
  __shared__ float rs2[2 * NS];
  __shared__ __align__(16) float wsh[2][2][WLD];
  const int tid = threadIdx.x;
  const int ic[3] = {g.n[0] / 2, g.n[1] / 2, g.n[2] / 2};
  const long long count = interior ? (long long)ic[0] * ic[1] * ic[2] : g.nverts;
  const long long item = blockIdx.x;
  if (item >= count) return;   // uniform over the block
  int vx, vy, vz;
  if (interior) {
    vx = 2 * (int)(item % ic[0]) + 1;
    vy = 2 * (int)((item / ic[0]) % ic[1]) + 1;
    vz = 2 * (int)(item / ((long long)ic[0] * ic[1])) + 1;
  } else {
    vx = (int)(item % g.nv[0]);
    vy = (int)((item / g.nv[0]) % g.nv[1]);
    vz = (int)(item / ((long long)g.nv[0] * g.nv[1]));
  }
  const long long v = (long long)vx + (long long)g.nv[0] * ((long long)vy + (long long)g.nv[1] * vz);
  const TS* W = inv + v * WSTRIDE;
  RowPair<TS> rp;
  rp.load(W, tid);
  for (int e = tid; e < NS; e += STAR_THREADS) {
    long long nd;
    const float val = star_node(g, vx, vy, vz, e, nd) ? r[(e / SN) * g.N + nd] : 0.f;
    rs2[e] = val;
    rs2[e + NS] = val;
  }
  float acc[STAR_ROWS];
#pragma unroll
  for (int k = 0; k < STAR_ROWS; ++k) acc[k] = 0.f;
  rp.store(&wsh[0][0][0], tid);
  __syncthreads();
  for (int pr = 0; pr < WT / 2; ++pr) {
    const int cur = pr & 1;
    if (pr + 1 < WT / 2) rp.load(W + (long long)(pr + 1) * 2 * WLD, tid);   // in flight during this pair
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = 2 * pr + h;
      const float* wr = wsh[cur][h];
#pragma unroll
      for (int k = 0; k < STAR_ROWS; ++k) {
        const int i = tid + STAR_THREADS * k;
        if (i < NS) {
          acc[k] += wr[i] * rs2[i + t];
          if (t > 0) {
            const int m = i - t < 0 ? i - t + NS : i - t;   // row m = i - t (mod NS) holds A(m, i)
            acc[k] += wr[m] * rs2[m];
          }
        }
      }
    }
    if (pr + 1 < WT / 2) rp.store(&wsh[cur ^ 1][0][0], tid);
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < STAR_ROWS; ++k) {
    const int i = tid + STAR_THREADS * k;
    if (i >= NS) continue;
    if (!interior) {
      out[v * NS + i] = acc[k];
    } else {
      long long nd;
      if (star_node(g, vx, vy, vz, i, nd)) {
        float* o = out + (i / SN) * g.N + nd;
        *o = mode == 2 ? *o - acc[k] : acc[k];
      }
    }
  }
}

// the wrapped rows in bfloat16, rounded to nearest from the FP64 packed diagonals
__global__ void k_qk3_wrap16(long long nverts, int pstride, const double* __restrict__ inv64,
                             __nv_bfloat16* __restrict__ inv16) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nverts * WSTRIDE) return;
  const long long v = e / WSTRIDE;
  const int r = (int)(e % WSTRIDE), t = r / WLD, i = r % WLD;
  double val = 0.0;
  if (i < NS) {
    const int j = i + t;
    const double* S = inv64 + v * pstride;
    val = j < NS ? S[diag_start(NS, t) + i] : S[diag_start(NS, NS - t) + (j - NS)];
  }
  inv16[e] = __double2bfloat16(val);
}

// the wrapped FP32 rows from the FP64 packed diagonals (loading caller-supplied inverses)
__global__ void k_qk3_wrap32(long long nverts, int pstride, const double* __restrict__ inv64,
                             float* __restrict__ inv32) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nverts * WSTRIDE) return;
  const long long v = e / WSTRIDE;
  const int r = (int)(e % WSTRIDE), t = r / WLD, i = r % WLD;
  float val = 0.f;
  if (i < NS) {
    const int j = i + t;
    const double* S = inv64 + v * pstride;
    val = (float)(j < NS ? S[diag_start(NS, t) + i] : S[diag_start(NS, NS - t) + (j - NS)]);
  }
  inv32[e] = val;
}

// z(node) = sum over the (up to 8) stars containing the node (vertices v with
// |i - 3v| <= 2 per axis), fixed order; 0 at Dirichlet nodes; divided by den[0] when given
template <typename T>
__global__ void k_qk3_star_gather(Geom g, const T* __restrict__ sc, T* __restrict__ z, const T* __restrict__ den) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * g.N) return;
  const int comp = (int)(t / g.N);
  const long long nd = t - comp * g.N;
  const int i = (int)(nd % g.nn[0]);
  const long long rr = nd / g.nn[0];
  const int j = (int)(rr % g.nn[1]), k = (int)(rr / g.nn[1]);
  if (bnd_node(g, i, j, k)) { z[t] = T(0); return; }
  int vs[3][2], os[3][2], m[3];
  const int ijk[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    const int v0 = ijk[a] / K, r = ijk[a] - K * v0;
    m[a] = 0;
    vs[a][m[a]] = v0; os[a][m[a]++] = r;
    if (r != 0) { vs[a][m[a]] = v0 + 1; os[a][m[a]++] = r - K; }
  }
  T acc = T(0);
  for (int c = 0; c < m[2]; ++c)
    for (int b = 0; b < m[1]; ++b)
      for (int a = 0; a < m[0]; ++a) {
        const long long v = (long long)vs[0][a] + (long long)g.nv[0] * ((long long)vs[1][b] + (long long)g.nv[1] * vs[2][c]);
        const int e = comp * SN + (os[0][a] + K - 1) + S1 * (os[1][b] + K - 1) + S1 * S1 * (os[2][c] + K - 1);
        acc += sc[v * NS + e];
      }
  if (den) acc = den[0] != T(0) ? acc / den[0] : T(0);
  z[t] = acc;
}

// ---------------------------------------------------------------------------
// transfers: P_H (the coarse Q3 basis at the fine nodes, tensor product of 1D weights;
// each fine node belongs to the coarse cell min(f div 6, nc - 1) per axis) and its
// transpose, by per-coarse-cell contractions; fine Dirichlet rows and coarse Dirichlet
// columns are zero
// ---------------------------------------------------------------------------

// xf = P_H xc (and xadd += xf): per coarse cell (one CTA) its 64 coarse values (zero at
// Dirichlet coarse nodes) contracted with the 1D weights along x, y, z into the 7^3 fine
// values, each written by the cell that owns the fine node (the owner rule of the
// restriction below; Dirichlet fine nodes get zero)
template <typename T>
__global__ void __launch_bounds__(128) k_qk3_prolong_cells(Geom gc, Geom gf, const T* __restrict__ xc,
                                                           T* __restrict__ xf, T* __restrict__ xadd) {
  __shared__ T u[3][NB];
  __shared__ T t1[3][NF * N1 * N1];
  __shared__ T t2[3][NF * NF * N1];
  __shared__ T pw[NF][N1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long cell = blockIdx.x;
  const int cx = (int)(cell % gc.n[0]), cy = (int)((cell / gc.n[0]) % gc.n[1]),
            cz = (int)(cell / ((long long)gc.n[0] * gc.n[1]));
  if (tid < NF * N1) pw[tid / N1][tid % N1] = Tab<T>::pw(tid / N1, tid % N1);
  for (int e = tid; e < 3 * NB; e += nt) {
    const int c = e / NB, a = e % NB;
    const int I = K * cx + a % N1, J = K * cy + (a / N1) % N1, Kz = K * cz + a / (N1 * N1);
    u[c][a] = bnd_node(gc, I, J, Kz) ? T(0) : xc[c * gc.N + node_id(gc, I, J, Kz)];
  }
  __syncthreads();
  for (int e = tid; e < 3 * NF * N1 * N1; e += nt) {   // x: (ax, ay, az) -> (fx, ay, az)
    const int c = e / (NF * N1 * N1), r = e % (NF * N1 * N1), fx = r % NF, yz = r / NF;
    T acc = T(0);
#pragma unroll
    for (int ax = 0; ax < N1; ++ax) acc += pw[fx][ax] * u[c][ax + N1 * yz];
    t1[c][r] = acc;
  }
  __syncthreads();
  for (int e = tid; e < 3 * NF * NF * N1; e += nt) {   // y: (fx, ay, az) -> (fx, fy, az)
    const int c = e / (NF * NF * N1), r = e % (NF * NF * N1), fx = r % NF, fy = (r / NF) % NF, az = r / (NF * NF);
    T acc = T(0);
#pragma unroll
    for (int ay = 0; ay < N1; ++ay) acc += pw[fy][ay] * t1[c][fx + NF * (ay + N1 * az)];
    t2[c][r] = acc;
  }
  __syncthreads();
  for (int e = tid; e < 3 * NF * NF * NF; e += nt) {   // z: (fx, fy, az) -> (fx, fy, fz), owned nodes
    const int c = e / (NF * NF * NF), r = e % (NF * NF * NF), fxy = r % (NF * NF), fx = r % NF, fy = fxy / NF,
              fz = r / (NF * NF);
    if ((fx == NF - 1 && cx != gc.n[0] - 1) || (fy == NF - 1 && cy != gc.n[1] - 1) ||
        (fz == NF - 1 && cz != gc.n[2] - 1))
      continue;
    T acc = T(0);
#pragma unroll
    for (int az = 0; az < N1; ++az) acc += pw[fz][az] * t2[c][fxy + NF * NF * az];
    const int i = 2 * K * cx + fx, j = 2 * K * cy + fy, k = 2 * K * cz + fz;
    const T v = bnd_node(gf, i, j, k) ? T(0) : acc;
    const long long fn = c * gf.N + node_id(gf, i, j, k);
    xf[fn] = v;
    if (xadd) xadd[fn] += v;
  }
}

// rc = P_H^T (rf - sub) in two steps.  Per coarse cell (one CTA): the 7^3 fine values it
// owns (a fine node on the face shared with the next coarse cell belongs to that cell;
// Dirichlet fine nodes are zero) contracted with the 1D weights along x, y, z into the
// cell's 64 node values, staged per cell; then k_qk3_gather sums the staged values of the
// cells containing each coarse node (zero at Dirichlet nodes).  A fine node outside the
// cells of a coarse node lies where that node's basis function vanishes, so the owner
// rule gives exactly P_H^T.
constexpr int RS_THREADS = 128;
template <typename T>
__global__ void __launch_bounds__(RS_THREADS) k_qk3_restrict_cells(Geom gc, Geom gf, const T* __restrict__ rf,
                                                                   const T* __restrict__ sub, T* __restrict__ stage) {
  __shared__ T v[3][NF * NF * NF];
  __shared__ T t1[3][N1 * NF * NF];
  __shared__ T t2[3][N1 * N1 * NF];
  __shared__ T pw[NF][N1];
  const int tid = threadIdx.x;
  const long long cell = blockIdx.x;
  const int cx = (int)(cell % gc.n[0]), cy = (int)((cell / gc.n[0]) % gc.n[1]),
            cz = (int)(cell / ((long long)gc.n[0] * gc.n[1]));
  if (tid < NF * N1) pw[tid / N1][tid % N1] = Tab<T>::pw(tid / N1, tid % N1);
  for (int e = tid; e < NF * NF * NF; e += RS_THREADS) {
    const int fx = e % NF, fy = (e / NF) % NF, fz = e / (NF * NF);
    const bool own = (fx < NF - 1 || cx == gc.n[0] - 1) && (fy < NF - 1 || cy == gc.n[1] - 1) &&
                     (fz < NF - 1 || cz == gc.n[2] - 1);
    const int i = 2 * K * cx + fx, j = 2 * K * cy + fy, k = 2 * K * cz + fz;
    const bool use = own && !bnd_node(gf, i, j, k);
    const long long nd = node_id(gf, i, j, k);
    for (int c = 0; c < 3; ++c) {
      const long long fn = c * gf.N + nd;
      v[c][e] = use ? (sub ? rf[fn] - sub[fn] : rf[fn]) : T(0);
    }
  }
  __syncthreads();
  for (int e = tid; e < 3 * N1 * NF * NF; e += RS_THREADS) {   // x: (fx, fy, fz) -> (ax, fy, fz)
    const int c = e / (N1 * NF * NF), r = e % (N1 * NF * NF), ax = r % N1, yz = r / N1;
    T acc = T(0);
#pragma unroll
    for (int fx = 0; fx < NF; ++fx) acc += pw[fx][ax] * v[c][fx + NF * yz];
    t1[c][r] = acc;
  }
  __syncthreads();
  for (int e = tid; e < 3 * N1 * N1 * NF; e += RS_THREADS) {   // y: (ax, fy, fz) -> (ax, ay, fz)
    const int c = e / (N1 * N1 * NF), r = e % (N1 * N1 * NF), ax = r % N1, ay = (r / N1) % N1, fz = r / (N1 * N1);
    T acc = T(0);
#pragma unroll
    for (int fy = 0; fy < NF; ++fy) acc += pw[fy][ay] * t1[c][ax + N1 * (fy + NF * fz)];
    t2[c][r] = acc;
  }
  __syncthreads();
  for (int e = tid; e < 3 * NB; e += RS_THREADS) {              // z: (ax, ay, fz) -> (ax, ay, az)
    const int c = e / NB, a = e % NB, axy = a % (N1 * N1), az = a / (N1 * N1);
    T acc = T(0);
#pragma unroll
    for (int fz = 0; fz < NF; ++fz) acc += pw[fz][az] * t2[c][axy + N1 * N1 * fz];
    stage[(cell * 3 + c) * NB + a] = acc;
  }
}

}  // namespace qk3

// ---------------------------------------------------------------------------
// entry points, called by qk.cu's dispatchers for 3D levels
// ---------------------------------------------------------------------------
void qk3_tables() { qk3::ensure_tables(); }

void qk3_apply(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y, const void* p_in,
               void* p_out, cudaStream_t s) {
  if (prec == PREC_F64) qk3::apply_t<double>(L, mode, gamma, x, y, p_in, p_out, s);
  else qk3::apply_t<float>(L, mode, gamma, x, y, p_in, p_out, s);
}

void qk3_apply_epi(const LevelDev& L, int prec, double gamma, const void* x, void* y, const ApplyEpi& e,
                   cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  if (prec == PREC_F64) qk3::apply_epi_t<double>(L, gamma, x, y, e, s, e0, e1);
  else qk3::apply_epi_t<float>(L, gamma, x, y, e, s, e0, e1);
}

void qk3_load_vector(const LevelDev& L, const double* f_qp, double* F, cudaStream_t s) {
  const long long tot = L.g.ncells * 3 * qk3::NB;
  qk3::k_qk3_load<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.g, f_qp, (double*)L.ebuf);
  qk3::k_qk3_gather<double><<<(unsigned)((3 * L.g.N + 255) / 256), 256, 0, s>>>(L.g, (const double*)L.ebuf, nullptr,
                                                                               F, 0, 1);
  count_launch(2);
}

void qk3_mass_setup(const LevelDev& L, double gamma, int w_mu, int variant, double* winv64, float* winv32, double* S,
                    DevStatus* st, cudaStream_t s) {
  qk3::k_qk3_mass<<<(unsigned)((L.g.ncells + 127) / 128), 128, 0, s>>>(L.g, gamma, L.mu64, w_mu, variant, winv64,
                                                                       winv32, S, st);
  count_launch(1);
}

// CTAs of the star setup (each holds one 375 x 376 FP64 star matrix in the workspace)
int qk3_setup_ctas(long long nverts) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = 2LL * sms;
  return (int)(nverts < want ? nverts : want);
}
size_t qk3_setup_ws_doubles(int ctas) { return (size_t)ctas * qk3::NS * qk3::LDM; }
size_t qk3_star32_floats() { return qk3::WSTRIDE; }

void qk3_derive32(const LevelDev& L, cudaStream_t s) {
  const long long tot = L.g.nverts * qk3::WSTRIDE;
  qk3::k_qk3_wrap32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.g.nverts, L.pstride, L.inv64, L.inv32);
  count_launch(1);
  if (L.inv16) {
    qk3::k_qk3_wrap16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.g.nverts, L.pstride, L.inv64,
                                                                   (__nv_bfloat16*)L.inv16);
    count_launch(1);
  }
}

void qk3_patch_setup(const LevelDev& L, double gamma, DevStatus* st, cudaStream_t s, int df64) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(qk3::k_qk3_star_setup<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)qk3::SETUP_SMEM);
    cudaFuncSetAttribute(qk3::k_qk3_star_setup<DF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)qk3::SETUP_SMEM);
    attr = true;
  }
  const int ctas = L.qk_ws_ctas < L.g.nverts ? L.qk_ws_ctas : (int)L.g.nverts;
  if (df64)
    qk3::k_qk3_star_setup<DF64><<<(unsigned)ctas, qk3::SETUP_THREADS, qk3::SETUP_SMEM, s>>>(
        L.g, gamma, L.mu64, L.winv64, L.qk_ws, L.inv64, L.inv32, L.pstride, st);
  else
    qk3::k_qk3_star_setup<double><<<(unsigned)ctas, qk3::SETUP_THREADS, qk3::SETUP_SMEM, s>>>(
        L.g, gamma, L.mu64, L.winv64, L.qk_ws, L.inv64, L.inv32, L.pstride, st);
  count_launch(1);
  if (L.inv16) {   // ALS_STORE_BF16: the rows again in bfloat16, from the FP64 inverses
    const long long tot = L.g.nverts * qk3::WSTRIDE;
    qk3::k_qk3_wrap16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(L.g.nverts, L.pstride, L.inv64,
                                                                   (__nv_bfloat16*)L.inv16);
    count_launch(1);
  }
}

void qk3_patch_smooth(const LevelDev& L, int prec, const void* r, void* z, void* scratch, const void* den,
                      cudaStream_t s) {
  const unsigned b3 = (unsigned)((3 * L.g.N + 255) / 256);
  const unsigned nv = (unsigned)L.g.nverts;
  if (prec == PREC_F64) {
    qk3::k_qk3_star_apply<double><<<nv, qk3::STAR_THREADS, 0, s>>>(L.g, L.inv64, L.pstride, 0, 0, (const double*)r,
                                                                   (double*)scratch);
    qk3::k_qk3_star_gather<double><<<b3, 256, 0, s>>>(L.g, (const double*)scratch, (double*)z, (const double*)den);
  } else {
    if (L.inv16)
      qk3::k_qk3_star_apply_w<__nv_bfloat16><<<nv, qk3::STAR_THREADS, 0, s>>>(
          L.g, (const __nv_bfloat16*)L.inv16, 0, 0, (const float*)r, (float*)scratch);
    else
      qk3::k_qk3_star_apply_w<float><<<nv, qk3::STAR_THREADS, 0, s>>>(L.g, L.inv32, 0, 0, (const float*)r,
                                                                      (float*)scratch);
    qk3::k_qk3_star_gather<float><<<b3, 256, 0, s>>>(L.g, (const float*)scratch, (float*)z, (const float*)den);
  }
  count_launch(2);
}

void qk3_interior_solve(const LevelDev& fine, int prec, const void* in, void* out, int subtract, cudaStream_t s) {
  const long long nc = (long long)(fine.g.n[0] / 2) * (fine.g.n[1] / 2) * (fine.g.n[2] / 2);
  const size_t es = prec == PREC_F64 ? 8 : 4;
  if (!subtract) cudaMemsetAsync(out, 0, es * 3 * fine.g.N, s);
  if (prec == PREC_F64)
    qk3::k_qk3_star_apply<double><<<(unsigned)nc, qk3::STAR_THREADS, 0, s>>>(
        fine.g, fine.inv64, fine.pstride, 1, subtract ? 2 : 1, (const double*)in, (double*)out);
  else
    if (fine.inv16)
      qk3::k_qk3_star_apply_w<__nv_bfloat16><<<(unsigned)nc, qk3::STAR_THREADS, 0, s>>>(
          fine.g, (const __nv_bfloat16*)fine.inv16, 1, subtract ? 2 : 1, (const float*)in, (float*)out);
    else
      qk3::k_qk3_star_apply_w<float><<<(unsigned)nc, qk3::STAR_THREADS, 0, s>>>(
          fine.g, fine.inv32, 1, subtract ? 2 : 1, (const float*)in, (float*)out);
  count_launch(1);
}

void qk3_prolong(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf, cudaStream_t s,
                 void* xadd) {
  const unsigned nc = (unsigned)coarse.g.ncells;
  if (prec == PREC_F64)
    qk3::k_qk3_prolong_cells<double><<<nc, 128, 0, s>>>(coarse.g, fine.g, (const double*)xc, (double*)xf,
                                                        (double*)xadd);
  else
    qk3::k_qk3_prolong_cells<float><<<nc, 128, 0, s>>>(coarse.g, fine.g, (const float*)xc, (float*)xf,
                                                       (float*)xadd);
  count_launch(1);
}

// the coarse level's per-cell output buffer stages the cell contributions (the coarse
// level's own applies, which use it too, come after the restriction on the stream)
void qk3_restrict(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc, cudaStream_t s,
                  const void* sub) {
  const unsigned nc = (unsigned)coarse.g.ncells, b = (unsigned)((3 * coarse.g.N + 255) / 256);
  if (prec == PREC_F64) {
    qk3::k_qk3_restrict_cells<double><<<nc, qk3::RS_THREADS, 0, s>>>(coarse.g, fine.g, (const double*)rf,
                                                                    (const double*)sub, (double*)coarse.ebuf);
    qk3::k_qk3_gather<double><<<b, 256, 0, s>>>(coarse.g, (const double*)coarse.ebuf, nullptr, (double*)rc, 0, 0);
  } else {
    qk3::k_qk3_restrict_cells<float><<<nc, qk3::RS_THREADS, 0, s>>>(coarse.g, fine.g, (const float*)rf,
                                                                   (const float*)sub, (float*)coarse.ebuf);
    qk3::k_qk3_gather<float><<<b, 256, 0, s>>>(coarse.g, (const float*)coarse.ebuf, nullptr, (float*)rc, 0, 0);
  }
  count_launch(2);
}

}  // namespace als
