// K7: coarse-grid solve (Sec. 6.1 uses a sparse direct solver on the coarsest
// level; here the coarsest A_gamma is small and dense-factored on the GPU).
//
// Setup: the free-dof block of the coarsest A_gamma is formed column by column
// by applying the matrix-free operator to unit vectors, factored by a
// right-looking FP64 Cholesky (one column per step), and its inverse
// L^-T L^-1 is formed by one triangular solve pair per column.  Each V-cycle
// then applies the stored FP64 inverse as a dense matrix-vector product.
#include "krylov.h"
#include "level.h"

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

__global__ void k_extract(Geom g, int nfree, long long len, const double* __restrict__ Y, double* __restrict__ A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nfree * nfree) return;
  const int col = (int)(t / nfree), row = (int)(t % nfree);
  // column `col` of A is A e_col; stored row-major A[row][col]
  A[(long long)row * nfree + col] = Y[(long long)col * len + free_dof(g, row)];
}

__global__ void k_chol_col(int n, int k, double* __restrict__ A, DevStatus* st) {
  __shared__ double piv;
  if (threadIdx.x == 0) {
    double d = A[(long long)k * n + k];
    if (!(d > 0.0)) { report(st, 4 /* ALS_ENOTSPD */, -1 - (long long)k); d = 1.0; }
    piv = sqrt(d);
    A[(long long)k * n + k] = piv;
  }
  __syncthreads();
  for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(long long)i * n + k] /= piv;
}

__global__ void k_chol_update(int n, int k, double* __restrict__ A) {
  const int i = k + 1 + blockIdx.x;
  if (i >= n) return;
  const double lik = A[(long long)i * n + k];
  for (int j = k + 1 + threadIdx.x; j <= i; j += blockDim.x) A[(long long)i * n + j] -= lik * A[(long long)j * n + k];
}

// column j of (L L^T)^-1: forward then backward substitution, one warp per column
__global__ void k_chol_inverse(int n, const double* __restrict__ L, double* __restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  // X stored row-major; column j written as X[i*n + j]
  for (int i = 0; i < j; ++i)
    if (lane == 0) X[(long long)i * n + j] = 0.0;
  __syncwarp();
  for (int i = j; i < n; ++i) {
    double acc = 0.0;
    for (int k = j + lane; k < i; k += 32) acc += L[(long long)i * n + k] * X[(long long)k * n + j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) X[(long long)i * n + j] = ((i == j ? 1.0 : 0.0) - acc) / L[(long long)i * n + i];
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = 0.0;
    for (int k = i + 1 + lane; k < n; k += 32) acc += L[(long long)k * n + i] * X[(long long)k * n + j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) X[(long long)i * n + j] = (X[(long long)i * n + j] - acc) / L[(long long)i * n + i];
    __syncwarp();
  }
}

int coarse_alloc(const LevelDev& L, CoarseDev* C) {
  const Geom& g = L.g;
  const int nfree = count_free(g);
  const long long len = g.N * g.dim;
  C->nfree = nfree;
  if (cudaMalloc(&C->X, sizeof(double) * nfree * len) != cudaSuccess) return 2;
  if (cudaMalloc(&C->Y, sizeof(double) * nfree * len) != cudaSuccess) return 2;
  if (cudaMalloc(&C->A, sizeof(double) * nfree * nfree) != cudaSuccess) return 2;
  if (cudaMalloc(&C->inv, sizeof(double) * nfree * nfree) != cudaSuccess) return 2;
  return 0;
}

// Forms and factors the coarsest A_gamma with the current coefficients (stream-ordered).
void coarse_setup(const LevelDev& L, double gamma, CoarseDev* C, DevStatus* st, cudaStream_t s) {
  const Geom& g = L.g;
  const int nfree = C->nfree;
  const long long len = g.N * g.dim;
  double *X = C->X, *Y = C->Y, *A = C->A;
  const long long tot = (long long)nfree * len;
  k_unit_columns<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g, nfree, len, X);
  op_apply_multi(L, gamma, X, Y, nfree, len, s);
  const long long tot2 = (long long)nfree * nfree;
  k_extract<<<(unsigned)((tot2 + 255) / 256), 256, 0, s>>>(g, nfree, len, Y, A);
  for (int k = 0; k < nfree; ++k) {
    k_chol_col<<<1, 256, 0, s>>>(nfree, k, A, st);
    if (k + 1 < nfree) k_chol_update<<<nfree - k - 1, 128, 0, s>>>(nfree, k, A);
  }
  k_chol_inverse<<<(nfree + 3) / 4, 128, 0, s>>>(nfree, A, C->inv);
  count_launch(3 + 2 * nfree);
}

template <typename TV>
__global__ void k_coarse_apply(Geom g, int nfree, const double* __restrict__ inv, const TV* __restrict__ b,
                               TV* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nfree) return;
  double acc = 0.0;
  for (int c = lane; c < nfree; c += 32) acc += inv[(long long)r * nfree + c] * (double)b[free_dof(g, c)];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[free_dof(g, r)] = (TV)acc;
}

void coarse_apply(const LevelDev& L, const CoarseDev& C, int prec, const void* b, void* x, cudaStream_t s) {
  const long long len = L.g.N * L.g.dim;
  cudaMemsetAsync(x, 0, len * (prec == PREC_F64 ? 8 : 4), s);
  const unsigned blocks = (unsigned)((C.nfree + 7) / 8);
  if (prec == PREC_F64) k_coarse_apply<double><<<blocks, 256, 0, s>>>(L.g, C.nfree, C.inv, (const double*)b, (double*)x);
  else k_coarse_apply<float><<<blocks, 256, 0, s>>>(L.g, C.nfree, C.inv, (const float*)b, (float*)x);
  count_launch(1);
}

void coarse_free(CoarseDev* C) {
  for (double** p : {&C->inv, &C->X, &C->Y, &C->A}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
}

}  // namespace als
