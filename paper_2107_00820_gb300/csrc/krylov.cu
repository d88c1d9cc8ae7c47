// K8/K9/K11: vector kernels, Krylov bookkeeping on the device, Schur block apply.
//
// All reductions use a fixed grid and a fixed combination order, so results
// are bitwise reproducible from run to run.  Small dense work (Givens
// rotations of the Hessenberg matrices, triangular solves) runs in
// single-thread kernels so that no step of a solve needs the host.
#include <math.h>

#include <atomic>

#include "batch.cuh"
#include "krylov.h"
#include "level.h"
#include "reduce.cuh"
#include "pdl.cuh"

namespace als {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launch(long long n) { g_launches += n; }

static constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs (two-pass sums of the pressure space)

template <typename T>
__global__ void k_axpby(long long n, double a, const T* __restrict__ x, double b, T* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + (b == 0.0 ? 0.0 : b * (double)y[i]));
}

template <typename T>
__global__ void k_axpy_dev(long long n, const double* __restrict__ a, double sign, const T* __restrict__ x,
                           T* __restrict__ y) {
  const T s = (T)(sign * a[0]);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += s * x[i];
}

template <typename S, typename D>
__global__ void k_cast(long long n, const S* __restrict__ x, D* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (D)x[i];
}

template <typename T>
__global__ void k_scale_dev(long long n, const double* __restrict__ num, const double* __restrict__ den,
                            const T* __restrict__ x, T* __restrict__ y, int sqrt_den) {
  const double dn = den ? (sqrt_den ? sqrt(fmax(den[0], 0.0)) : den[0]) : 1.0;
  const double f = (num ? num[0] : 1.0);
  const T s = (T)(dn != 0.0 ? f / dn : 0.0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = s * x[i];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;  // valid in thread 0
}

// out[j] = V_j . w for j < k
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_multidot(long long n, int k, const T* __restrict__ V, long long ld,
                                                          const T* __restrict__ w, double* __restrict__ partial,
                                                          double* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int j0 = 0; j0 < k; j0 += KMAXB) {
    const int kk = (k - j0) < KMAXB ? (k - j0) : KMAXB;
    double acc[KMAXB];
#pragma unroll
    for (int jj = 0; jj < KMAXB; ++jj) acc[jj] = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const double wi = (double)w[i];
#pragma unroll
      for (int jj = 0; jj < KMAXB; ++jj)
        if (jj < kk) acc[jj] += (double)V[(long long)(j0 + jj) * ld + i] * wi;
    }
    block_partials(acc, kk, partial + 1 + (long long)blockIdx.x * k + j0);
  }
  if (last_block(partial)) finish_sums(partial, k, out);
}

// w <- w + sign * sum_j V_j h_j, and nrm2 = w . w of the updated w
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_multiaxpy_norm(long long n, int k, const T* __restrict__ V,
                                                                long long ld, const double* __restrict__ h,
                                                                double sign, T* __restrict__ w,
                                                                double* __restrict__ partial,
                                                                double* __restrict__ nrm2) {
  double acc2 = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += (double)V[(long long)j * ld + i] * h[j];
    const T wn = (T)((double)w[i] + sign * acc);
    w[i] = wn;
    acc2 += (double)wn * (double)wn;
  }
  double a8[KMAXB] = {acc2};
  block_partials(a8, 1, partial + 1 + blockIdx.x);
  if (last_block(partial)) finish_sums(partial, 1, nrm2);
}

template <typename T>
__global__ void k_multiaxpy(long long n, int k, const T* __restrict__ V, long long ld, const double* __restrict__ h,
                            double sign, T* __restrict__ w) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += (double)V[(long long)j * ld + i] * h[j];
    w[i] = (T)((double)w[i] + sign * acc);
  }
}

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 8) b = 152LL * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

void vec_axpby(int prec, long long n, double a, const void* x, double b, void* y, cudaStream_t s) {
  if (prec == PREC_F64) k_axpby<double><<<grid_for(n), 256, 0, s>>>(n, a, (const double*)x, b, (double*)y);
  else k_axpby<float><<<grid_for(n), 256, 0, s>>>(n, a, (const float*)x, b, (float*)y);
  count_launch(1);
}

void vec_axpy_dev(int prec, long long n, const double* a, double sign, const void* x, void* y, cudaStream_t s) {
  if (prec == PREC_F64) k_axpy_dev<double><<<grid_for(n), 256, 0, s>>>(n, a, sign, (const double*)x, (double*)y);
  else k_axpy_dev<float><<<grid_for(n), 256, 0, s>>>(n, a, sign, (const float*)x, (float*)y);
  count_launch(1);
}

void vec_cast(long long n, const void* src, int src_prec, void* dst, int dst_prec, cudaStream_t s) {
  if (src_prec == PREC_F64 && dst_prec == PREC_F32) {
    k_cast<double, float><<<grid_for(n), 256, 0, s>>>(n, (const double*)src, (float*)dst);
    count_launch(1);
  } else if (src_prec == PREC_F32 && dst_prec == PREC_F64) {
    k_cast<float, double><<<grid_for(n), 256, 0, s>>>(n, (const float*)src, (double*)dst);
    count_launch(1);
  } else
    cudaMemcpyAsync(dst, src, n * (src_prec == PREC_F64 ? 8 : 4), cudaMemcpyDeviceToDevice, s);
}

void vec_zero(int prec, long long n, void* x, cudaStream_t s) {
  cudaMemsetAsync(x, 0, n * (prec == PREC_F64 ? 8 : 4), s);
}

// ticket counter slot + partial sums of up to RED_MAX_BLOCKS blocks for k columns
size_t multidot_partial_doubles(int k) { return (size_t)RED_MAX_BLOCKS * (size_t)k + 1; }

static unsigned red_grid(long long n) { return red_blocks(n); }

void vec_multidot(int prec, long long n, int k, const void* V, long long ld, const void* w, double* out,
                  double* partial, cudaStream_t s) {
  if (prec == PREC_F64)
    k_multidot<double><<<red_grid(n), RED_THREADS, 0, s>>>(n, k, (const double*)V, ld, (const double*)w, partial, out);
  else
    k_multidot<float><<<red_grid(n), RED_THREADS, 0, s>>>(n, k, (const float*)V, ld, (const float*)w, partial, out);
  count_launch(1);
}

void vec_multiaxpy_norm(int prec, long long n, int k, const void* V, long long ld, const double* h, double sign,
                        void* w, double* partial, double* nrm2, cudaStream_t s) {
  if (prec == PREC_F64)
    k_multiaxpy_norm<double><<<red_grid(n), RED_THREADS, 0, s>>>(n, k, (const double*)V, ld, h, sign, (double*)w,
                                                                   partial, nrm2);
  else
    k_multiaxpy_norm<float><<<red_grid(n), RED_THREADS, 0, s>>>(n, k, (const float*)V, ld, h, sign, (float*)w,
                                                                  partial, nrm2);
  count_launch(1);
}

void vec_multiaxpy(int prec, long long n, int k, const void* V, long long ld, const double* h, void* w,
                   cudaStream_t s, double sign) {
  if (prec == PREC_F64)
    k_multiaxpy<double><<<grid_for(n), 256, 0, s>>>(n, k, (const double*)V, ld, h, sign, (double*)w);
  else
    k_multiaxpy<float><<<grid_for(n), 256, 0, s>>>(n, k, (const float*)V, ld, h, sign, (float*)w);
  count_launch(1);
}

void vec_multiaxpy(int prec, long long n, int k, const void* V, long long ld, const double* h, void* w,
                   cudaStream_t s) {
  vec_multiaxpy(prec, n, k, V, ld, h, w, s, -1.0);
}

void vec_scale_dev(int prec, long long n, const double* num, const double* den, const void* x, void* y,
                   cudaStream_t s, int sqrt_den) {
  if (prec == PREC_F64)
    k_scale_dev<double><<<grid_for(n), 256, 0, s>>>(n, num, den, (const double*)x, (double*)y, sqrt_den);
  else k_scale_dev<float><<<grid_for(n), 256, 0, s>>>(n, num, den, (const float*)x, (float*)y, sqrt_den);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// GMRES(s) smoother steps with an unnormalised stored basis (see GmresDev)
// ---------------------------------------------------------------------------
// Each thread handles PER entries spaced RED_THREADS apart, with all loads of
// its entries issued before any arithmetic; the grid then has about n / (256 PER)
// blocks, which keeps the ticket counter of the single-launch reduction cold
// (same-address atomics serialise: several thousand blocks cost microseconds).
// Column loops are unrolled to KMAXB with predicates.  In FP32 the arithmetic
// and all sums run in float, and so does the small GMRES bookkeeping (the state
// array holds elements of the smoother's precision).
constexpr int GM_PER = 4;

// V0 = b, |b|^2 -> gmres_start
// (bx, nb: the block's index and the blocks of this reduction, see batch.cuh)
template <typename T>
__device__ __forceinline__ void gm_start_body(unsigned bx, unsigned nb, unsigned n, const T* __restrict__ b,
                                              T* __restrict__ V0, double* __restrict__ partial, GmresDev sd) {
  __shared__ T nrm2_s[1];
  const GmresView<T> st = gmres_view<T>(sd);
  T* rows = reinterpret_cast<T*>(partial + 1);
  const unsigned base = bx * (RED_THREADS * GM_PER) + threadIdx.x;
  pdl_wait();
  T v[GM_PER];
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
    v[q] = i < n ? b[i] : T(0);
  }
  T acc[KMAXB] = {T(0)};
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
    if (i < n) V0[i] = v[q];
    acc[0] += v[q] * v[q];
  }
  pdl_trigger();
  block_partials<T, T>(acc, 1, rows + bx);
  if (last_block(partial, nb)) {
    finish_sums_n<T>(partial, 1, nrm2_s, nullptr, (int)nb);
    if (threadIdx.x == 0) gmres_start(st, nrm2_s[0]);
  }
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_gm_start(unsigned n, const T* __restrict__ b, T* __restrict__ V0,
                                                          double* __restrict__ partial, GmresDev sd) {
  gm_start_body<T>(blockIdx.x, gridDim.x, n, b, V0, partial, sd);
}

// Gram-Schmidt update of the new column w = V_{j+1} against columns 0..j with the
// coefficients H[0..j][j] / hn[i], then |w|^2 -> gmres_step(j)
template <typename T>
__device__ __forceinline__ void gm_orth_body(unsigned bx, unsigned nb, unsigned n, int j, const T* __restrict__ V,
                                             long long ld, double* __restrict__ partial, GmresDev sd) {
  __shared__ T coef[KMAXB];
  __shared__ T nrm2_s[1];
  const GmresView<T> st = gmres_view<T>(sd);
  T* rows = reinterpret_cast<T*>(partial + 1);
  T* w = const_cast<T*>(V) + (long long)(j + 1) * ld;
  const unsigned base = bx * (RED_THREADS * GM_PER) + threadIdx.x;
  T a[GM_PER];
  T vc[GM_PER][KMAXB];
  // columns 0..j come from earlier kernels of the chain (complete before this launch
  // began): read through L2 before the wait; column j+1 and H come from the predecessor
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
#pragma unroll
    for (int c = 0; c < KMAXB; ++c) vc[q][c] = (i < n && c <= j) ? __ldcg(V + (long long)c * ld + i) : T(0);
  }
  pdl_wait();
  const T* hcol = st.H + (long long)j * st.ldh;
  if ((int)threadIdx.x <= j)
    coef[threadIdx.x] = st.hn[threadIdx.x] != T(0) ? hcol[threadIdx.x] / st.hn[threadIdx.x] : T(0);
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
    a[q] = i < n ? w[i] : T(0);
  }
  __syncthreads();
  T acc[KMAXB] = {T(0)};
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
#pragma unroll
    for (int c = 0; c < KMAXB; ++c)
      if (c <= j) a[q] -= vc[q][c] * coef[c];
    if (i < n) w[i] = a[q];
    acc[0] += a[q] * a[q];
  }
  pdl_trigger();
  block_partials<T, T>(acc, 1, rows + bx);
  if (last_block(partial, nb)) {
    finish_sums_n<T>(partial, 1, nrm2_s, nullptr, (int)nb);
    if (threadIdx.x == 0) {
      gmres_step(st, j, nrm2_s[0]);
      if (j == st.m - 2) gmres_coeffs(st, j + 1);   // last step: the update's coefficients, once
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_gm_orth(unsigned n, int j, const T* __restrict__ V, long long ld,
                                                         double* __restrict__ partial, GmresDev sd) {
  gm_orth_body<T>(blockIdx.x, gridDim.x, n, j, V, ld, partial, sd);
}

// x = (x_zero ? 0 : x) + sum_j Z_j y_j with y = R^-1 g, and, if t != NULL, the
// GMRES residual  t = r0 - A Z y = sum_i u_i v_i,  u = Q^T (g[k] e_k)  from the
// Arnoldi relation (Q = product of the Givens rotations), no operator apply.  y and
// u were formed once by the last block of the last k_gm_orth (gmres_coeffs).
template <typename T>
__device__ __forceinline__ void gm_update_body(unsigned bx, unsigned n, int k, const T* __restrict__ Z,
                                               const T* __restrict__ V, long long ld, GmresDev sd,
                                               T* __restrict__ x, int x_zero, T* __restrict__ t) {
  __shared__ T y[KMAXB], u[KMAXB + 1];
  const GmresView<T> st = gmres_view<T>(sd);
  const unsigned base = bx * (RED_THREADS * GM_PER) + threadIdx.x;
  // Z, x and V_0..V_{k-1} come from earlier kernels of the chain (complete before this
  // launch began): read through L2 before the wait; V_k and the coefficients come
  // from the predecessor (the last Gram-Schmidt step)
  T zc[GM_PER][KMAXB], xa[GM_PER];
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
#pragma unroll
    for (int c = 0; c < KMAXB; ++c) zc[q][c] = (i < n && c < k) ? __ldcg(Z + (long long)c * ld + i) : T(0);
    xa[q] = (i < n && !x_zero) ? __ldcg(x + i) : T(0);
  }
  pdl_wait();
  // coefficients from the last k_gm_orth of the cycle (gmres_coeffs), cast to T
  if ((int)threadIdx.x < k) y[threadIdx.x] = st.yu[threadIdx.x];
  else if ((int)threadIdx.x <= 2 * k && t) u[threadIdx.x - k] = st.yu[threadIdx.x];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < GM_PER; ++q) {
    const unsigned i = base + q * RED_THREADS;
    if (i >= n) break;
    T a = xa[q];
#pragma unroll
    for (int c = 0; c < KMAXB; ++c)
      if (c < k) a += zc[q][c] * y[c];
    x[i] = a;
  }
  if (t) {
#pragma unroll
    for (int q = 0; q < GM_PER; ++q) {
      const unsigned i = base + q * RED_THREADS;
      if (i >= n) break;
      T vc[KMAXB + 1];
#pragma unroll
      for (int c = 0; c <= KMAXB; ++c) vc[c] = c <= k ? V[(long long)c * ld + i] : T(0);
      T r = T(0);
#pragma unroll
      for (int c = 0; c <= KMAXB; ++c)
        if (c <= k) r += vc[c] * u[c];
      t[i] = r;
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_gm_update(unsigned n, int k, const T* __restrict__ Z,
                                                           const T* __restrict__ V, long long ld, GmresDev sd,
                                                           T* __restrict__ x, int x_zero, T* __restrict__ t) {
  gm_update_body<T>(blockIdx.x, n, k, Z, V, ld, sd, x, x_zero, t);
}

static unsigned full_grid(long long n) {
  return (unsigned)((n + RED_THREADS * GM_PER - 1) / (RED_THREADS * GM_PER));
}

void gm_start(int prec, long long n, const void* b, void* V0, double* partial, const GmresDev& st, cudaStream_t s) {
  if (prec == PREC_F64)
    launch_pdl(k_gm_start<double>, full_grid(n), RED_THREADS, 0, s, (unsigned)n, (const double*)b, (double*)V0, partial, st);
  else
    launch_pdl(k_gm_start<float>, full_grid(n), RED_THREADS, 0, s, (unsigned)n, (const float*)b, (float*)V0, partial, st);
  count_launch(1);
}

void gm_orth(int prec, long long n, int j, const void* V, long long ld, double* partial, const GmresDev& st,
             cudaStream_t s) {
  if (prec == PREC_F64)
    launch_pdl(k_gm_orth<double>, full_grid(n), RED_THREADS, 0, s, (unsigned)n, j, (const double*)V, ld, partial, st);
  else
    launch_pdl(k_gm_orth<float>, full_grid(n), RED_THREADS, 0, s, (unsigned)n, j, (const float*)V, ld, partial, st);
  count_launch(1);
}

void gm_update(int prec, long long n, int k, const void* Z, const void* V, long long ld, const GmresDev& st,
               void* x, int x_zero, void* t, cudaStream_t s) {
  if (prec == PREC_F64)
    launch_pdl(k_gm_update<double>, full_grid(n), RED_THREADS, 0, s, (unsigned)n, k, (const double*)Z, (const double*)V, ld,
                                                               st, (double*)x, x_zero, (double*)t);
  else
    launch_pdl(k_gm_update<float>, full_grid(n), RED_THREADS, 0, s, (unsigned)n, k, (const float*)Z, (const float*)V, ld,
                                                              st, (float*)x, x_zero, (float*)t);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// merged launches (batch.cuh): the same bodies, one launch for all instances
// ---------------------------------------------------------------------------
struct GmArgs {
  unsigned n;
  int j;
  const float* b;
  const float* Z;
  float* V;
  long long ld;
  double* partial;
  GmresDev st;
  float* x;
  int x_zero;
  float* t;
};

__global__ void __launch_bounds__(RED_THREADS) k_gm_start_b(const __grid_constant__ BatchTab<GmArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const GmArgs& a = tb.a[i];
  gm_start_body<float>(blockIdx.x - tb.start[i], tb.start[i + 1] - tb.start[i], a.n, a.b, a.V, a.partial, a.st);
}
__global__ void __launch_bounds__(RED_THREADS) k_gm_orth_b(const __grid_constant__ BatchTab<GmArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const GmArgs& a = tb.a[i];
  gm_orth_body<float>(blockIdx.x - tb.start[i], tb.start[i + 1] - tb.start[i], a.n, a.j, a.V, a.ld, a.partial, a.st);
}
__global__ void __launch_bounds__(RED_THREADS) k_gm_update_b(const __grid_constant__ BatchTab<GmArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const GmArgs& a = tb.a[i];
  gm_update_body<float>(blockIdx.x - tb.start[i], a.n, a.st.s, a.Z, a.V, a.ld, a.st, a.x, a.x_zero, a.t);
}

struct ZeroArgs {
  float* x;
  unsigned n;
};
__global__ void __launch_bounds__(256) k_zero_b(const __grid_constant__ BatchTab<ZeroArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const ZeroArgs& a = tb.a[i];
  pdl_wait();
  const unsigned e = (blockIdx.x - tb.start[i]) * 1024u + threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (e + 256u * q < a.n) a.x[e + 256u * q] = 0.f;
  pdl_trigger();
}

static int batch_gm(void (*k)(BatchTab<GmArgs>), const std::vector<BGmres>& items, cudaStream_t s) {
  std::vector<GmArgs> a;
  std::vector<unsigned> nb;
  for (const BGmres& it : items) {
    a.push_back(GmArgs{(unsigned)it.n, it.j, (const float*)it.b, (const float*)it.Z, (float*)it.V, it.ld, it.partial,
                       it.st, (float*)it.x, it.x_zero, (float*)it.t});
    nb.push_back(full_grid(it.n));
  }
  const int n = launch_batch(k, a, nb, RED_THREADS, 0, s);
  count_launch(n);
  return n;
}
int batch_gm_start(const std::vector<BGmres>& items, cudaStream_t s) { return batch_gm(k_gm_start_b, items, s); }
int batch_gm_orth(const std::vector<BGmres>& items, cudaStream_t s) { return batch_gm(k_gm_orth_b, items, s); }
int batch_gm_update(const std::vector<BGmres>& items, cudaStream_t s) { return batch_gm(k_gm_update_b, items, s); }

int batch_zero(const std::vector<BZero>& items, cudaStream_t s) {
  std::vector<ZeroArgs> a;
  std::vector<unsigned> nb;
  for (const BZero& it : items) {
    a.push_back(ZeroArgs{(float*)it.x, (unsigned)it.n});
    nb.push_back((unsigned)((it.n + 1023) / 1024));
  }
  const int n = launch_batch(k_zero_b, a, nb, 256, 0, s);
  count_launch(n);
  return n;
}

// workspace of the smoother's fused reductions: one partial row of KMAXB per block
size_t gmres_partial_doubles(long long n) {
  return (size_t)((n + RED_THREADS - 1) / RED_THREADS) * KMAXB + 1;   // covers every grid used
}

// ---------------------------------------------------------------------------
// small dense work on the device
// ---------------------------------------------------------------------------
__global__ void k_sqrt(const double* __restrict__ in, double* __restrict__ out) { out[0] = sqrt(fmax(in[0], 0.0)); }

void dev_sqrt(const double* in, double* out, cudaStream_t s) { k_sqrt<<<1, 1, 0, s>>>(in, out);
  count_launch(1); }

// h[0..k] += h2[0..k]; H[k+1][k] (stored at hcol[k+1]) = sqrt(nrm2)
__global__ void k_hess_finish(int k, double* __restrict__ hcol, const double* __restrict__ h2,
                              const double* __restrict__ nrm2) {
  for (int i = 0; i <= k; ++i) hcol[i] += h2 ? h2[i] : 0.0;
  hcol[k + 1] = sqrt(fmax(nrm2[0], 0.0));
}

void dev_hess_finish(int k, double* hcol, const double* h2, const double* nrm2, cudaStream_t s) {
  k_hess_finish<<<1, 1, 0, s>>>(k, hcol, h2, nrm2);
  count_launch(1);
}

// Incremental Givens QR of the Hessenberg matrix of (F)GMRES.
// H is column-major with leading dimension ldh; column k has entries 0..k+1.
// State: cs, sn (rotations), g (rotated right-hand side, g[0] = beta initially).
// Writes |g[k+1]| (the residual norm of the least-squares problem) to res.
__global__ void k_givens_step(int k, double* __restrict__ H, int ldh, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, double* __restrict__ res) {
  double* h = H + (long long)k * ldh;
  for (int i = 0; i < k; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = h[k], b = h[k + 1];
  const double r = hypot(a, b);
  double c = 1.0, sv = 0.0;
  if (r > 0.0) { c = a / r; sv = b / r; }
  cs[k] = c; sn[k] = sv;
  h[k] = r; h[k + 1] = 0.0;
  g[k + 1] = -sv * g[k];
  g[k] = c * g[k];
  res[0] = fabs(g[k + 1]);
}

// column k of the Hessenberg matrix: h[0..k] += h2 (second Gram-Schmidt pass, optional),
// h[k+1] = sqrt(nrm2); then the Givens step as in k_givens_step
__global__ void k_hess_givens(int k, double* __restrict__ H, int ldh, const double* __restrict__ h2,
                              const double* __restrict__ nrm2, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, double* __restrict__ res) {
  double* h = H + (long long)k * ldh;
  if (h2)
    for (int i = 0; i <= k; ++i) h[i] += h2[i];
  h[k + 1] = sqrt(fmax(nrm2[0], 0.0));
  for (int i = 0; i < k; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = h[k], b = h[k + 1];
  const double r = hypot(a, b);
  double c = 1.0, sv = 0.0;
  if (r > 0.0) { c = a / r; sv = b / r; }
  cs[k] = c; sn[k] = sv;
  h[k] = r; h[k + 1] = 0.0;
  g[k + 1] = -sv * g[k];
  g[k] = c * g[k];
  res[0] = fabs(g[k + 1]);
}

void dev_hess_givens(int k, double* H, int ldh, const double* h2, const double* nrm2, double* cs, double* sn,
                     double* g, double* res, cudaStream_t s) {
  k_hess_givens<<<1, 1, 0, s>>>(k, H, ldh, h2, nrm2, cs, sn, g, res);
  count_launch(1);
}

void dev_givens_step(int k, double* H, int ldh, double* cs, double* sn, double* g, double* res, cudaStream_t s) {
  k_givens_step<<<1, 1, 0, s>>>(k, H, ldh, cs, sn, g, res);
  count_launch(1);
}

// y = R^-1 g for the rotated (upper-triangular) k x k Hessenberg; a zero
// pivot (exact breakdown) drops that direction.
__global__ void k_backsolve(int k, const double* __restrict__ H, int ldh, const double* __restrict__ g,
                            double* __restrict__ y) {
  for (int i = k - 1; i >= 0; --i) {
    double acc = g[i];
    for (int j = i + 1; j < k; ++j) acc -= H[(long long)j * ldh + i] * y[j];
    const double d = H[(long long)i * ldh + i];
    y[i] = d != 0.0 ? acc / d : 0.0;
  }
}

void dev_backsolve(int k, const double* H, int ldh, const double* g, double* y, cudaStream_t s) {
  k_backsolve<<<1, 1, 0, s>>>(k, H, ldh, g, y);
  count_launch(1);
}

// g = (beta, 0, ...), where beta = sqrt(nrm2)
__global__ void k_init_g(int m, const double* __restrict__ nrm2, double* __restrict__ g, double* __restrict__ beta) {
  const double b = sqrt(fmax(nrm2[0], 0.0));
  beta[0] = b;
  g[0] = b;
  for (int i = 1; i < m; ++i) g[i] = 0.0;
}

void dev_init_g(int m, const double* nrm2, double* g, double* beta, cudaStream_t s) {
  k_init_g<<<1, 1, 0, s>>>(m, nrm2, g, beta);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// pressure space: Schur block apply and constant-mode projection
// ---------------------------------------------------------------------------
__global__ void k_schur(long long ncells, int npr, const double* __restrict__ S, const double* __restrict__ t,
                        double* __restrict__ z) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int i = 0; i < npr; ++i) {
    double acc = 0.0;
    for (int j = 0; j < npr; ++j) acc += S[(c * npr + i) * npr + j] * t[c * npr + j];
    z[c * npr + i] = -acc;
  }
}

void schur_apply(long long ncells, int npr, const double* S, const double* t, double* z, cudaStream_t s) {
  k_schur<<<(unsigned)((ncells + 255) / 256), 256, 0, s>>>(ncells, npr, S, t, z);
  count_launch(1);
}

__global__ void k_slot0_sum(long long ncells, int npr, const double* __restrict__ p, double* __restrict__ partial) {
  __shared__ double sh[RED_THREADS / 32];
  double acc = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (long long)gridDim.x * blockDim.x)
    acc += p[c * npr];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[1 + blockIdx.x] = s;
}

__global__ void k_slot0_sub(long long ncells, int npr, const double* __restrict__ partial, int nb, double* __restrict__ p) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[1 + b];
  const double mean = s / (double)ncells;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (long long)gridDim.x * blockDim.x)
    p[c * npr] -= mean;
}

// p <- p - (n.p / n.n) n with n = 1 on the constant-basis slot of every cell
void project_constant(long long ncells, int npr, double* p, double* partial, cudaStream_t s) {
  k_slot0_sum<<<RED_BLOCKS, RED_THREADS, 0, s>>>(ncells, npr, p, partial);
  k_slot0_sub<<<grid_for(ncells), 256, 0, s>>>(ncells, npr, partial, RED_BLOCKS, p);
  count_launch(2);
}

}  // namespace als

namespace als {

// ---------------------------------------------------------------------------
// Schur-complement blocks of Eq. (P1P2), variant P1, one (d+1)x(d+1) FP64 block
// per cell: S_K = M_K(1/mu)^-1 + gamma M_K^-1 with
// [M_K(1/mu)]_ab = sum_q |J| w_q mu_q^-1 psi_a(x_q) psi_b(x_q) (Eq. (inv-visc-mass))
// and M_K = |K| diag(1, 1/3, ..).  The small SPD block is inverted through
// its Cholesky factor.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_schur_setup(Geom g, double gamma, const double* __restrict__ mu, double* __restrict__ S,
                              DevStatus* st, int variant, double* __restrict__ winv64, float* __restrict__ winv32) {
  constexpr int NPR = DIM + 1, NB = DIM == 2 ? 9 : 27;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncells) return;
  double wdet = 1.0, vol = 1.0;
  for (int k = 0; k < DIM; ++k) { wdet *= 0.5 * g.h[k]; vol *= g.h[k]; }
  double M[NPR][NPR];
  for (int a = 0; a < NPR; ++a)
    for (int b = 0; b < NPR; ++b) M[a][b] = 0.0;
  for (int q = 0; q < NB; ++q) {
    const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    double psi[NPR];
    psi[0] = 1.0; psi[1] = Ref<double>::G(qx); psi[2] = Ref<double>::G(qy);
    if (DIM == 3) psi[3] = Ref<double>::G(qz);
    const double w = wdet * Ref<double>::W(qx) * Ref<double>::W(qy) * (DIM == 3 ? Ref<double>::W(qz) : 1.0) /
                     mu[c * NB + q];
    for (int a = 0; a < NPR; ++a)
      for (int b = 0; b < NPR; ++b) M[a][b] += w * psi[a] * psi[b];
  }
  // Cholesky M = L L^T, then X = L^-1, inverse = X^T X
  double Lm[NPR][NPR] = {};
  for (int j = 0; j < NPR; ++j) {
    double d = M[j][j];
    for (int k = 0; k < j; ++k) d -= Lm[j][k] * Lm[j][k];
    if (!(d > 0.0)) { report(st, 4, c); d = 1.0; }
    Lm[j][j] = sqrt(d);
    for (int i = j + 1; i < NPR; ++i) {
      double v = M[i][j];
      for (int k = 0; k < j; ++k) v -= Lm[i][k] * Lm[j][k];
      Lm[i][j] = v / Lm[j][j];
    }
  }
  double X[NPR][NPR] = {};
  for (int i = 0; i < NPR; ++i)
    for (int j = 0; j <= i; ++j) {
      double acc = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) acc -= Lm[i][k] * X[k][j];
      X[i][j] = acc / Lm[i][i];
    }
  for (int i = 0; i < NPR; ++i)
    for (int j = 0; j < NPR; ++j) {
      double acc = 0.0;                     // [M_K(1/mu)^-1]_ij
      for (int k = (i > j ? i : j); k < NPR; ++k) acc += X[k][i] * X[k][j];
      if (winv64) winv64[(c * NPR + i) * NPR + j] = acc;
      if (winv32) winv32[(c * NPR + i) * NPR + j] = (float)acc;
      if (!S) continue;
      if (variant == 0) {                   // P1: M_p(1/mu)^-1 + gamma M_p^-1
        if (i == j) acc += gamma * (i == 0 ? 1.0 : 3.0) / vol;
      } else {                              // P2: (1 + gamma) M_p(1/mu)^-1
        acc *= 1.0 + gamma;
      }
      S[(c * NPR + i) * NPR + j] = acc;
    }
}

void schur_setup(const Geom& g, double gamma, const double* mu, double* S, DevStatus* st, cudaStream_t s,
                 int variant, double* winv64, float* winv32) {
  const unsigned b = (unsigned)((g.ncells + 127) / 128);
  if (g.dim == 2) k_schur_setup<2><<<b, 128, 0, s>>>(g, gamma, mu, S, st, variant, winv64, winv32);
  else k_schur_setup<3><<<b, 128, 0, s>>>(g, gamma, mu, S, st, variant, winv64, winv32);
  count_launch(1);
}

// keep_boundary = 1: y = x on boundary nodes, 0 inside; keep_boundary = 0: the converse
__global__ void k_bnd_mask(Geom g, const double* __restrict__ x, double* __restrict__ y, int keep_boundary) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N * g.dim) return;
  const long long nd = t % g.N;
  const int i = (int)(nd % g.nn[0]);
  const long long r = nd / g.nn[0];
  const int j = (int)(r % g.nn[1]);
  const int k = (int)(r / g.nn[1]);
  const bool b = on_boundary(g, i, j, k);
  y[t] = (b == (keep_boundary != 0)) ? x[t] : 0.0;
}

void bnd_mask(const Geom& g, const double* x, double* y, int keep_boundary, cudaStream_t s) {
  const long long tot = g.N * g.dim;
  k_bnd_mask<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g, x, y, keep_boundary);
  count_launch(1);
}

// out = gamma W^-1 r2 with W = M_p = |K| diag(1, 1/3, ..) on every cell
__global__ void k_winv(long long ncells, int npr, double scale0, double scale1, const double* __restrict__ r2,
                       double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells * npr) return;
  out[t] = r2[t] * ((t % npr) == 0 ? scale0 : scale1);
}

__global__ void k_winv_block(long long ncells, int npr, double gamma, const double* __restrict__ winv,
                             const double* __restrict__ r2, double* __restrict__ out) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  for (int i = 0; i < npr; ++i) {
    double acc = 0.0;
    for (int j = 0; j < npr; ++j) acc += winv[(c * npr + i) * npr + j] * r2[c * npr + j];
    out[c * npr + i] = gamma * acc;
  }
}

void winv_scale(const Geom& g, double gamma, const double* r2, double* out, cudaStream_t s, const double* winv,
                int npr) {
  if (winv) {
    k_winv_block<<<(unsigned)((g.ncells + 255) / 256), 256, 0, s>>>(g.ncells, npr > 0 ? npr : g.dim + 1, gamma, winv, r2,
                                                                    out);
    count_launch(1);
    return;
  }
  double vol = 1.0;
  for (int k = 0; k < g.dim; ++k) vol *= g.h[k];
  const long long tot = g.ncells * (g.dim + 1);
  k_winv<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g.ncells, g.dim + 1, gamma / vol, 3.0 * gamma / vol, r2, out);
  count_launch(1);
}

}  // namespace als

namespace als {

// Smallest positive entry of x (the bit patterns of positive doubles order like their
// values, so an unsigned 64-bit atomic minimum finds it); entries <= 0 or NaN are skipped.
// *out_bits must hold the bits of +inf before the first call.
__global__ void k_min_positive(long long n, const double* __restrict__ x, unsigned long long* __restrict__ out_bits) {
  unsigned long long best = 0x7ff0000000000000ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (v > 0.0) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(v);
      best = b < best ? b : best;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_down_sync(0xffffffffu, best, o);
    best = other < best ? other : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMin(out_bits, best);
}

void vec_min_positive(long long n, const double* x, unsigned long long* out_bits, cudaStream_t s) {
  if (n <= 0) return;
  const long long want = (n + 255) / 256, blocks = want < 152LL * 8 ? want : 152LL * 8;
  k_min_positive<<<(unsigned)blocks, 256, 0, s>>>(n, x, out_bits);
  count_launch(1);
}

}  // namespace als
