// K7: coarse-grid solve (Sec. 5.1 uses a sparse direct solver on the coarsest
// level; here the coarsest A_gamma is small and dense-inverted on the GPU).
//
// Setup: the free-dof block of the coarsest A_gamma is formed column by column
// by applying the matrix-free operator to unit vectors and inverted (in FP64, or in
// double-float arithmetic for the mixed cycle) by a blocked symmetric sweep (the operator of the patch setup, applied to 64-wide
// pivot blocks): per block K, S = A_KK^-1 by a one-CTA sweep of the diagonal
// block, U = A_{:K} S, A_RR -= A_{RK} U_R^T on the upper triangle of tiles, and
// the pivot row/column set to U (A_KK to -S).  After every block the matrix holds
// -A^-1.  A is SPD, so every pivot is a Schur complement and positive.  Each
// V-cycle then applies the stored inverse as a dense matrix-vector product.
#include "batch.cuh"
#include "cell.cuh"
#include "df64.cuh"
#include "krylov.h"
#include "level.h"
#include "pdl.cuh"

#include <algorithm>

namespace als {

__device__ __forceinline__ long long free_dof(const Geom& g, int f) {
  const int ni = g.nn[0] - 2, nj = g.nn[1] - 2, nk = g.dim == 3 ? g.nn[2] - 2 : 1;
  const long long nint = (long long)ni * nj * nk;
  const int c = (int)(f / nint);
  const long long m = f % nint;
  const int i = (int)(m % ni) + 1;
  const int j = (int)((m / ni) % nj) + 1;
  const int k = g.dim == 3 ? (int)(m / ((long long)ni * nj)) + 1 : 0;
  return (long long)c * g.N + node_id(g, i, j, k);
}

static int count_free(const Geom& g) {
  long long n = (long long)(g.nn[0] - 2) * (g.nn[1] - 2) * (g.dim == 3 ? g.nn[2] - 2 : 1);
  return (int)(n * g.dim);
}

__global__ void k_unit_columns(Geom g, int nfree, long long len, double* __restrict__ X) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nfree * len) return;
  const int col = (int)(t / len);
  const long long dof = t % len;
  X[t] = (dof == free_dof(g, col)) ? 1.0 : 0.0;
}

constexpr int CT = 64;   // tile width of the blocked sweep

// The blocked sweep runs in R = FP64, or DF64 (FP32 pairs, about 48 bits, see
// df64.cuh) when only the FP32 cycle needs the inverse; the buffers A, P, U, S hold
// elements of R (8 bytes either way) and the inverse is written in FP64.

// column `col` of A is A e_col; stored row-major in the padded matrix (npad columns)
template <typename R>
__global__ void k_extract(Geom g, int nfree, int npad, long long len, const double* __restrict__ Y,
                          R* __restrict__ A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nfree * nfree) return;
  const int col = (int)(t / nfree), row = (int)(t % nfree);
  A[(long long)row * npad + col] = RealOps<R>::from(Y[(long long)col * len + free_dof(g, row)]);
}

// identity on the padding rows/columns (their blocks stay decoupled)
template <typename R>
__global__ void k_pad_diag(int nfree, int npad, R* __restrict__ A) {
  const int i = nfree + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) A[(long long)i * npad + i] = RealOps<R>::from(1.0);
}

// P[r][c] = A(r, p*CT + c) from the upper triangle of tiles
template <typename R>
__global__ void k_panel_gather(int npad, int p, const R* __restrict__ A, R* __restrict__ P) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)npad * CT) return;
  const int r = (int)(t / CT), c = (int)(t % CT), k = p * CT + c;
  const bool upper = r <= k;
  P[t] = upper ? A[(long long)r * npad + k] : A[(long long)k * npad + r];
}

// S = D^-1 for the diagonal block D = P[p*CT .. p*CT+CT) by the symmetric sweep
// in shared memory (one CTA of 1024 threads, the block is on the setup's critical path);
// a non-positive pivot is reported as ALS_ENOTSPD.
// Every thread of the pivot column forms 1/pivot itself (no wait on one thread).
template <typename R>
__global__ void __launch_bounds__(1024) k_diag_sweep(int p, const R* __restrict__ P, R* __restrict__ S,
                                                    DevStatus* st) {
  using O = RealOps<R>;
  __shared__ R D[CT][CT + 1];
  __shared__ R col[CT], q[CT];
  const int tid = threadIdx.x;
  const R zero = O::from(0.0), one = O::from(1.0);
  for (int e = tid; e < CT * CT; e += blockDim.x) D[e / CT][e % CT] = P[(long long)(p * CT + e / CT) * CT + e % CT];
  __syncthreads();
  for (int kk = 0; kk < CT; ++kk) {
    R d = D[kk][kk];
    if (!(d > 0.f)) {
      if (tid == 0) report(st, 4 /* ALS_ENOTSPD */, -1 - (long long)(p * CT + kk));
      d = one;
    }
    const R dinv = one / d;
    if (tid < CT) {
      const R c = tid == kk ? zero : D[tid][kk];
      col[tid] = c;
      q[tid] = c * dinv;
    }
    __syncthreads();
    for (int e = tid; e < CT * CT; e += blockDim.x) {
      const int i = e / CT, j = e % CT;
      if (i != kk && j != kk) D[i][j] = O::sub_prod(D[i][j], q[i], col[j]);
      else if (i == kk && j == kk) D[i][j] = -dinv;
      else D[i][j] = q[i == kk ? j : i];
    }
    __syncthreads();
  }
  for (int e = tid; e < CT * CT; e += blockDim.x) S[e] = -D[e / CT][e % CT];
}

// 64x64 output tile out = X_tile * Y (Y 64x64 row-major) or X_tile * Y_tile^T, 4x4 per thread
template <typename R>
__device__ __forceinline__ void tile_mma(const R (*Xs)[CT + 1], const R (*Ys)[CT + 1], bool yt, R (&acc)[4][4],
                                         int r0, int c0) {
  using O = RealOps<R>;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = O::from(0.0);
  for (int k = 0; k < CT; ++k) {
    R a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = Xs[r0 + 16 * i][k];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = yt ? Ys[c0 + 16 * j][k] : Ys[k][c0 + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = O::add_prod(acc[i][j], a[i], b[j]);
  }
}

// U[rows of tile blockIdx.x] = P[those rows] S
template <typename R>
__global__ void __launch_bounds__(256) k_panel_mul(const R* __restrict__ P, const R* __restrict__ S,
                                                   R* __restrict__ U) {
  extern __shared__ double smc[];
  R (*Ps)[CT + 1] = reinterpret_cast<R (*)[CT + 1]>(smc);
  R (*Ss)[CT + 1] = reinterpret_cast<R (*)[CT + 1]>(smc + CT * (CT + 1));
  const int tid = threadIdx.x;
  const long long r0 = (long long)blockIdx.x * CT;
  for (int e = tid; e < CT * CT; e += blockDim.x) {
    Ps[e / CT][e % CT] = P[(r0 + e / CT) * CT + e % CT];
    Ss[e / CT][e % CT] = S[e];
  }
  __syncthreads();
  R acc[4][4];
  const int tr = tid / 16, tc = tid % 16;
  tile_mma<R>(Ps, Ss, false, acc, tr, tc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) U[(r0 + tr + 16 * i) * CT + tc + 16 * j] = acc[i][j];
}

// A[I][J] -= P[I] U[J]^T for the upper tiles I <= J outside the pivot row/column p
template <typename R>
__global__ void __launch_bounds__(256) k_sym_update(int npad, int nt, int p, const R* __restrict__ P,
                                                    const R* __restrict__ U, R* __restrict__ A) {
  int b = blockIdx.x, I = 0;
  while (b >= nt - I) { b -= nt - I; ++I; }
  const int J = I + b;
  if (I == p || J == p) return;
  extern __shared__ double smc[];
  R (*Ps)[CT + 1] = reinterpret_cast<R (*)[CT + 1]>(smc);
  R (*Us)[CT + 1] = reinterpret_cast<R (*)[CT + 1]>(smc + CT * (CT + 1));
  const int tid = threadIdx.x;
  for (int e = tid; e < CT * CT; e += blockDim.x) {
    Ps[e / CT][e % CT] = P[((long long)I * CT + e / CT) * CT + e % CT];
    Us[e / CT][e % CT] = U[((long long)J * CT + e / CT) * CT + e % CT];
  }
  __syncthreads();
  R acc[4][4];
  const int tr = tid / 16, tc = tid % 16;
  tile_mma<R>(Ps, Us, true, acc, tr, tc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      R& a = A[((long long)I * CT + tr + 16 * i) * npad + (long long)J * CT + tc + 16 * j];
      a = RealOps<R>::add(a, -acc[i][j]);
    }
}

// pivot row/column p of the upper triangle: A(r, K) = U(r) for r outside K, A_KK = -S
template <typename R>
__global__ void k_panel_write(int npad, int p, const R* __restrict__ U, const R* __restrict__ S,
                              R* __restrict__ A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)npad * CT) return;
  const int r = (int)(t / CT), c = (int)(t % CT), k = p * CT + c, I = r / CT;
  if (I < p) A[(long long)r * npad + k] = U[t];
  else if (I > p) A[(long long)k * npad + r] = U[t];
  else A[(long long)r * npad + k] = -S[(r - p * CT) * CT + c];
}

// inv = -(swept matrix) on the free block, both triangles, in FP64
template <typename R>
__global__ void k_finalize(int nfree, int npad, const R* __restrict__ A, double* __restrict__ inv) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nfree * nfree) return;
  const int r = (int)(t / nfree), c = (int)(t % nfree);
  inv[t] = -RealOps<R>::to_double(r <= c ? A[(long long)r * npad + c] : A[(long long)c * npad + r]);
}

int coarse_alloc(const LevelDev& L, CoarseDev* C) {
  const Geom& g = L.g;
  const int nfree = count_free(g);
  const long long len = g.N * g.dim;
  C->nfree = nfree;
  if (cudaMalloc(&C->X, sizeof(double) * nfree * len) != cudaSuccess) return 2;
  if (cudaMalloc(&C->Y, sizeof(double) * nfree * len) != cudaSuccess) return 2;
  const int npad = (nfree + CT - 1) / CT * CT;
  C->npad = npad;
  if (cudaMalloc(&C->A, sizeof(double) * npad * npad) != cudaSuccess) return 2;
  if (cudaMalloc(&C->inv, sizeof(double) * nfree * nfree) != cudaSuccess) return 2;
  if (cudaMalloc(&C->P, sizeof(double) * npad * CT) != cudaSuccess) return 2;
  if (cudaMalloc(&C->U, sizeof(double) * npad * CT) != cudaSuccess) return 2;
  if (cudaMalloc(&C->S, sizeof(double) * CT * CT) != cudaSuccess) return 2;
  return 0;
}

template <typename R>
static void coarse_sweep(const LevelDev& L, CoarseDev* C, DevStatus* st, cudaStream_t s) {
  const Geom& g = L.g;
  const int nfree = C->nfree;
  const long long len = g.N * g.dim;
  R* A = reinterpret_cast<R*>(C->A);
  R* P = reinterpret_cast<R*>(C->P);
  R* U = reinterpret_cast<R*>(C->U);
  R* S = reinterpret_cast<R*>(C->S);
  const long long tot2 = (long long)nfree * nfree;
  const int npad = C->npad, nt = npad / CT;
  cudaMemsetAsync(A, 0, sizeof(R) * npad * npad, s);   // all-zero bits are 0 in both types
  if (npad > nfree) k_pad_diag<R><<<(npad - nfree + 127) / 128, 128, 0, s>>>(nfree, npad, A);
  k_extract<R><<<(unsigned)((tot2 + 255) / 256), 256, 0, s>>>(g, nfree, npad, len, C->Y, A);
  const size_t smem2 = sizeof(R) * 2 * CT * (CT + 1);
  cudaFuncSetAttribute(k_panel_mul<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  cudaFuncSetAttribute(k_sym_update<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  const unsigned pblocks = (unsigned)(((long long)npad * CT + 255) / 256);
  for (int p = 0; p < nt; ++p) {
    k_panel_gather<R><<<pblocks, 256, 0, s>>>(npad, p, A, P);
    k_diag_sweep<R><<<1, 1024, 0, s>>>(p, P, S, st);   // 4 entries of the 64x64 block per thread
    k_panel_mul<R><<<nt, 256, smem2, s>>>(P, S, U);
    k_sym_update<R><<<nt * (nt + 1) / 2, 256, smem2, s>>>(npad, nt, p, P, U, A);
    k_panel_write<R><<<pblocks, 256, 0, s>>>(npad, p, U, S, A);
  }
  k_finalize<R><<<(unsigned)((tot2 + 255) / 256), 256, 0, s>>>(nfree, npad, A, C->inv);
  count_launch(2 + (npad > nfree ? 1 : 0) + 5LL * nt);
}

// Forms and factors the coarsest A_gamma with the current coefficients (stream-ordered).
// df64: the sweep in double-float arithmetic (the inverse then carries about 48 bits).
static void coarse_apply_prepare(int nfree);

void coarse_setup(const LevelDev& L, double gamma, CoarseDev* C, DevStatus* st, cudaStream_t s, int df64) {
  const Geom& g = L.g;
  const int nfree = C->nfree;
  const long long len = g.N * g.dim;
  const long long tot = (long long)nfree * len;
  k_unit_columns<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g, nfree, len, C->X);
  if (L.k == 3) {   // the order-3 operator, one column at a time
    for (int c = 0; c < nfree; ++c)
      op_apply(L, PREC_F64, OP_VISC | OP_AL, gamma, C->X + (long long)c * len, C->Y + (long long)c * len, nullptr,
               nullptr, s);
  } else {
    op_apply_multi(L, gamma, C->X, C->Y, nfree, len, s);
  }
  count_launch(1);
  if (df64) coarse_sweep<DF64>(L, C, st, s);
  else coarse_sweep<double>(L, C, st, s);
  coarse_apply_prepare(nfree);
}

// 32-bit form of free_dof for the apply (vector lengths stay below 2^31)
__device__ __forceinline__ int free_dof32(const Geom& g, int f) {
  const int ni = g.nn[0] - 2, nj = g.nn[1] - 2, nk = g.dim == 3 ? g.nn[2] - 2 : 1;
  const int nint = ni * nj * nk;
  const int c = f / nint;
  const int m = f - c * nint;
  const int q = m / ni;
  const int i = m - q * ni + 1;
  const int j = g.dim == 3 ? q % nj + 1 : q + 1;
  const int k = g.dim == 3 ? q / nj + 1 : 0;
  return c * (int)g.N + i + g.nn[0] * (j + g.nn[1] * k);
}

// x_free = inv b_free, one warp per row.  STAGE: b at the free dofs is first
// gathered into shared memory (as double) by every block; otherwise (coarse
// problems too large for shared memory) each term reads b through the index map.
// Four independent FP64 partial sums per lane (dependent FP64 adds are slow on
// this GPU), combined in a fixed order.
template <typename TV, bool STAGE>
__device__ __forceinline__ void coarse_apply_body(unsigned bx, const Geom& g, int nfree, const double* __restrict__ inv,
                                                  const TV* __restrict__ b, TV* __restrict__ x) {
  extern __shared__ double bs[];
  pdl_wait();
  if (STAGE) {
    for (int c = threadIdx.x; c < nfree; c += blockDim.x) bs[c] = (double)b[free_dof32(g, c)];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int r = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nfree) return;
  const double* row = inv + (long long)r * nfree;
  auto bv = [&](int c) { return STAGE ? bs[c] : (double)b[free_dof32(g, c)]; };
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = lane;
  for (; c + 96 < nfree; c += 128) {
    a0 += row[c] * bv(c);
    a1 += row[c + 32] * bv(c + 32);
    a2 += row[c + 64] * bv(c + 64);
    a3 += row[c + 96] * bv(c + 96);
  }
  for (; c < nfree; c += 32) a0 += row[c] * bv(c);
  double acc = (a0 + a1) + (a2 + a3);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[free_dof32(g, r)] = (TV)acc;
}
template <typename TV, bool STAGE>
__global__ void __launch_bounds__(256) k_coarse_apply(Geom g, int nfree, const double* __restrict__ inv,
                                                      const TV* __restrict__ b, TV* __restrict__ x) {
  coarse_apply_body<TV, STAGE>(blockIdx.x, g, nfree, inv, b, x);
}

// merged launch (batch.cuh), FP32
struct CoarseArgs {
  Geom g;
  int nfree;
  const double* inv;
  const float* b;
  float* x;
};
template <bool STAGE>
__global__ void __launch_bounds__(256) k_coarse_apply_b(const __grid_constant__ BatchTab<CoarseArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const CoarseArgs& a = tb.a[i];
  coarse_apply_body<float, STAGE>(blockIdx.x - tb.start[i], a.g, a.nfree, a.inv, a.b, a.x);
}

constexpr size_t kCoarseStageMax = 200 * 1024;   // largest staged right-hand side (bytes)

// shared-memory opt-in of the staged apply, set at setup (never while a cycle is captured)
static void coarse_apply_prepare(int nfree) {
  const size_t smem = (size_t)nfree * sizeof(double);
  if (smem > 48 * 1024 && smem <= kCoarseStageMax) {
    cudaFuncSetAttribute(k_coarse_apply<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_coarse_apply<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
}

template <typename TV>
static void launch_coarse_apply(const LevelDev& L, const CoarseDev& C, const TV* b, TV* x, cudaStream_t s) {
  const unsigned blocks = (unsigned)((C.nfree + 7) / 8);
  const size_t smem = (size_t)C.nfree * sizeof(double);
  if (smem <= kCoarseStageMax) {   // opt-in above 48 KB set by coarse_apply_prepare at setup
    launch_pdl(k_coarse_apply<TV, true>, blocks, 256, smem, s, L.g, C.nfree, (const double*)C.inv, b, x);
  } else {
    launch_pdl(k_coarse_apply<TV, false>, blocks, 256, 0, s, L.g, C.nfree, (const double*)C.inv, b, x);
  }
}

void coarse_apply(const LevelDev& L, const CoarseDev& C, int prec, const void* b, void* x, cudaStream_t s) {
  const long long len = L.g.N * L.g.dim;
  cudaMemsetAsync(x, 0, len * (prec == PREC_F64 ? 8 : 4), s);
  if (prec == PREC_F64) launch_coarse_apply<double>(L, C, (const double*)b, (double*)x, s);
  else launch_coarse_apply<float>(L, C, (const float*)b, (float*)x, s);
  count_launch(1);
}

// merged: x = 0, then x_free = inv b_free for every item (the staged form when every
// item's right-hand side fits the staging limit, with room for the largest)
int batch_coarse_apply(const std::vector<BCoarse>& items, cudaStream_t s) {
  std::vector<BZero> z;
  std::vector<CoarseArgs> a;
  std::vector<unsigned> nb;
  int maxfree = 0;
  for (const BCoarse& it : items) {
    z.push_back(BZero{it.x, it.L->g.N * it.L->g.dim});
    a.push_back(CoarseArgs{it.L->g, it.C->nfree, (const double*)it.C->inv, (const float*)it.b, (float*)it.x});
    nb.push_back((unsigned)((it.C->nfree + 7) / 8));
    maxfree = std::max(maxfree, it.C->nfree);
  }
  const int nz = batch_zero(z, s);
  const size_t smem = (size_t)maxfree * sizeof(double);
  int n = 0;
  if (smem <= kCoarseStageMax) n = launch_batch(k_coarse_apply_b<true>, a, nb, 256, smem, s);
  else n = launch_batch(k_coarse_apply_b<false>, a, nb, 256, 0, s);
  count_launch(n);
  return nz + n;
}

// shared-memory opt-in of the merged staged apply (before any capture)
void batch_coarse_prepare() {
  cudaFuncSetAttribute(k_coarse_apply_b<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseStageMax);
}

void coarse_free(CoarseDev* C) {
  for (double** p : {&C->inv, &C->X, &C->Y, &C->A, &C->P, &C->U, &C->S}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

}  // namespace als
