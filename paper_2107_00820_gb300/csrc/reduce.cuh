// Single-launch, bitwise-reproducible reductions and the one-thread GMRES
// bookkeeping that runs in the epilogue of the last block of a reduction.
//
// Every block writes the partial sums of its columns to a workspace row, takes
// a ticket from a counter, and the block holding the last ticket adds the
// partials of all blocks in a fixed order (so the result does not depend on
// which block finished last) and resets the counter.  Workspace layout: slot 0
// is the counter, the partials [block][column] start at slot 1.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace als {

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1216;   // 8 x 152 SMs: one full wave at 256 threads per block
constexpr int KMAXB = 8;               // columns reduced together in registers

// blocks for a reduction over n entries: about `per_thread` entries per thread
inline unsigned red_blocks(long long n, int per_thread = 4) {
  long long b = (n + (long long)RED_THREADS * per_thread - 1) / ((long long)RED_THREADS * per_thread);
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// block partials of kk <= KMAXB columns: warp shuffles, one shared pass, written to row[0..kk).
// A is the accumulation type inside the block, R the type of the stored partials
// (double by default; the FP32 smoother keeps its sums in float throughout: FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU, with dependent
// FP64 latencies of 60-1100 cycles).
template <typename A, typename R = double>
__device__ __forceinline__ void block_partials(const A (&acc)[KMAXB], int kk, R* row) {
  __shared__ A sh[RED_THREADS / 32][KMAXB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < KMAXB; ++j) {
    if (j >= kk) break;
    A v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w][j] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < kk) {
    A v = A(0);
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += sh[i][threadIdx.x];
    row[threadIdx.x] = (R)v;
    __threadfence();   // the writers publish their partial before the block takes its ticket
  }
  __syncthreads();
}

// called right after block_partials (whose writers fenced their partials); nb = the
// blocks taking part in this reduction (the grid, or an instance's share of a merged launch)
__device__ __forceinline__ bool last_block(double* ws, unsigned nb) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) is_last = atomicAdd(reinterpret_cast<unsigned int*>(ws), 1u) == nb - 1;
  __syncthreads();
  return is_last;
}
__device__ __forceinline__ bool last_block(double* ws) { return last_block(ws, gridDim.x); }

// Run by every thread of the last block: out[j] = (sum over blocks of column j) / div[j]
// (div NULL: no division; div[j] == 0 gives 0).  The partials (type R, rows from
// ws + 1) are read through L2 (other blocks wrote them), each thread over a fixed
// strided subset, then one fixed block reduction per group of KMAXB columns, in R.
template <typename R = double>
__device__ __forceinline__ void finish_sums_n(double* ws, int k, R* out, const R* div, int nb) {
  if (threadIdx.x == 0) __threadfence();
  __syncthreads();
  const R* partial = reinterpret_cast<const R*>(ws + 1);
  for (int j0 = 0; j0 < k; j0 += KMAXB) {
    const int kk = (k - j0) < KMAXB ? (k - j0) : KMAXB;
    R acc[KMAXB];
#pragma unroll
    for (int j = 0; j < KMAXB; ++j) acc[j] = R(0);
#pragma unroll 4
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
      for (int j = 0; j < KMAXB; ++j)
        if (j < kk) acc[j] += __ldcg(partial + (long long)b * k + j0 + j);
    }
    __shared__ R tot[KMAXB];
    block_partials<R, R>(acc, kk, tot);
    if ((int)threadIdx.x < kk) {
      const int j = j0 + threadIdx.x;
      R v = tot[threadIdx.x];
      if (div) v = div[j] != R(0) ? v / div[j] : R(0);
      out[j] = v;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *reinterpret_cast<unsigned int*>(ws) = 0u;
}
template <typename R = double>
__device__ __forceinline__ void finish_sums(double* ws, int k, R* out, const R* div = nullptr) {
  finish_sums_n<R>(ws, k, out, div, (int)gridDim.x);
}

// ---------------------------------------------------------------------------
// GMRES(s) state on the device, in the smoother's precision T (column-major
// Hessenberg H, leading dim ldh).  The Krylov basis is stored unnormalised:
// column i holds hn[i] * v_i, where v_i is the orthonormal Arnoldi vector, and
// every consumer divides by hn[i].  Layout of the state array, in elements of T:
// H [ldh s] | cs [s] | sn [s] | g [s+1] | y [s] | res | beta | nrm2 | hn [s+1] | yu [2s+1].
// ---------------------------------------------------------------------------
struct GmresLayout {
  int s, ldh;
  int H, cs, sn, g, y, res, beta, nrm2, hn, yu, total;
  __host__ __device__ constexpr explicit GmresLayout(int steps)
      : s(steps), ldh(steps + 1), H(0), cs((steps + 1) * steps), sn(cs + steps), g(sn + steps), y(g + steps + 1),
        res(y + steps), beta(res + 1), nrm2(beta + 1), hn(nrm2 + 1), yu(hn + steps + 1), total(yu + 2 * steps + 1) {}
};

// host-side handle: the state array (elements of the smoother's precision) and s
struct GmresDev {
  void* base;
  int s;
};

template <typename T>
struct GmresView {
  T* H;
  int ldh;
  T* cs;
  T* sn;
  T* g;       // rotated right-hand side, length s + 1
  T* res;     // |g[k+1]| after step k
  T* hn;      // stored-column norms, length s + 1
  T* beta;    // |r0|
  int m;      // s + 1
  T* yu;      // after the last step: y = R^-1 g (s entries), then u = Q^T (g[s] e_s) / hn (s + 1)
};

template <typename T>
__host__ __device__ __forceinline__ GmresView<T> gmres_view(const GmresDev& d) {
  const GmresLayout L(d.s);
  T* b = static_cast<T*>(d.base);
  return GmresView<T>{b + L.H, L.ldh, b + L.cs, b + L.sn, b + L.g, b + L.res, b + L.hn, b + L.beta, d.s + 1, b + L.yu};
}

// start: beta = |r0|, g = (beta, 0, ...), hn[0] = beta   (one thread)
template <typename T>
__device__ __forceinline__ void gmres_start(const GmresView<T>& st, T nrm2) {
  const T b = sqrt(fmax(nrm2, T(0)));
  st.beta[0] = b;
  st.hn[0] = b;
  st.g[0] = b;
  for (int i = 1; i < st.m; ++i) st.g[i] = T(0);
}

// step k (k < KMAXB): H[k+1][k] = |w|, hn[k+1] = |w|, then the rotations of
// column k; all operands are loaded first so the chain runs in registers (one thread)
template <typename T>
__device__ __forceinline__ void gmres_step(const GmresView<T>& st, int k, T nrm2) {
  T* hg = st.H + (long long)k * st.ldh;
  T h[KMAXB + 1], cs[KMAXB], sn[KMAXB];
  for (int i = 0; i <= k; ++i) h[i] = hg[i];
  for (int i = 0; i < k; ++i) { cs[i] = st.cs[i]; sn[i] = st.sn[i]; }
  const T gk = st.g[k];
  const T hk1 = sqrt(fmax(nrm2, T(0)));
  h[k + 1] = hk1;
  for (int i = 0; i < k; ++i) {
    const T a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const T a = h[k], b = h[k + 1];
  const T r = hypot(a, b);
  T c = T(1), sv = T(0);
  if (r > T(0)) { c = a / r; sv = b / r; }
  h[k] = r;
  for (int i = 0; i <= k; ++i) hg[i] = h[i];
  hg[k + 1] = T(0);
  st.hn[k + 1] = hk1;
  st.cs[k] = c; st.sn[k] = sv;
  st.g[k + 1] = -sv * gk;
  st.g[k] = c * gk;
  st.res[0] = fabs(sv * gk);
}

// after step k - 1 (one thread): y = R^-1 g by back substitution on the rotated
// Hessenberg matrix, and u = Q^T (g[k] e_k) / hn (Q = product of the Givens
// rotations), so that x + Z y is the GMRES iterate and its residual is
// sum_i u_i (stored column i) by the Arnoldi relation.  Stored in st.yu.
template <typename T>
__device__ __forceinline__ void gmres_coeffs(const GmresView<T>& st, int k) {
  T Hs[KMAXB][KMAXB], gs[KMAXB + 1], cs[KMAXB], sn[KMAXB], hn[KMAXB + 1];
  for (int c = 0; c < k; ++c) {
    for (int r = 0; r <= c; ++r) Hs[r][c] = st.H[(long long)c * st.ldh + r];
    cs[c] = st.cs[c]; sn[c] = st.sn[c];
  }
  for (int c = 0; c <= k; ++c) { gs[c] = st.g[c]; hn[c] = st.hn[c]; }
  T ys[KMAXB];
  for (int i = k - 1; i >= 0; --i) {
    T a = gs[i];
    for (int c = i + 1; c < k; ++c) a -= Hs[i][c] * ys[c];
    ys[i] = Hs[i][i] != T(0) ? a / Hs[i][i] : T(0);
    st.yu[i] = ys[i];
  }
  T us[KMAXB + 1];
  for (int i = 0; i < k; ++i) us[i] = T(0);
  us[k] = gs[k];
  for (int i = k - 1; i >= 0; --i) {
    const T a = us[i], b = us[i + 1];
    us[i] = cs[i] * a - sn[i] * b;
    us[i + 1] = sn[i] * a + cs[i] * b;
  }
  for (int i = 0; i <= k; ++i) st.yu[k + i] = hn[i] != T(0) ? us[i] / hn[i] : T(0);
}

}  // namespace als
