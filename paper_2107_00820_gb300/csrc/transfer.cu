// K5: standard Q2 prolongation P_H and its transpose (Sec. 4.2).
//
// V_H is a subspace of V_h, so P_H is nested interpolation: a fine node at a
// coarse node takes its value; a fine node at a quarter point of a coarse cell
// takes the coarse quadratic there, 1D weights (3/8, 3/4, -1/8) at 1/4 and
// (-1/8, 3/4, 3/8) at 3/4, tensorised over the axes.  Dirichlet rows (fine
// boundary) and columns (coarse boundary) are zero.  Both directions are
// gathers (one thread per output value), so they need no atomics.
#include "batch.cuh"
#include "level.h"
#include "pdl.cuh"

namespace als {

// Fixed tap sets per axis (predicated, fully unrolled, so every load of an
// output issues at once).  A tap is used only if it lies inside the axis and off
// its Dirichlet ends: the boundary of the box is exactly the set of nodes with
// some coordinate at an end, so the per-axis test removes boundary rows/columns.

// fine node f (1D) -> three coarse taps (nc coarse nodes on the axis)
template <typename W>
__device__ __forceinline__ void prolong_taps(int f, int nc, int* m, W* w, bool* ok) {
  if ((f & 1) == 0) {
    m[0] = f >> 1; w[0] = W(1); m[1] = m[0]; w[1] = W(0); m[2] = m[0]; w[2] = W(0);
  } else {
    const int c = f >> 2;           // coarse cell
    const bool first = (f & 3) == 1;
    m[0] = 2 * c; m[1] = 2 * c + 1; m[2] = 2 * c + 2;
    w[0] = first ? W(0.375) : W(-0.125); w[1] = W(0.75); w[2] = first ? W(-0.125) : W(0.375);
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) ok[q] = w[q] != W(0) && m[q] >= 1 && m[q] <= nc - 2;
}

// coarse node m (1D) -> five fine taps of the transpose (nf fine nodes on the axis)
template <typename W>
__device__ __forceinline__ void restrict_taps(int m, int nf, int* f, W* w, bool* ok) {
  f[0] = 2 * m; w[0] = W(1);
  f[1] = 2 * m - 1; f[2] = 2 * m + 1;
  f[3] = 2 * m - 3; f[4] = 2 * m + 3;
  if (m & 1) { w[1] = w[2] = W(0.75); w[3] = w[4] = W(0); }
  else { w[1] = w[2] = W(0.375); w[3] = w[4] = W(-0.125); }
#pragma unroll
  for (int q = 0; q < 5; ++q) ok[q] = w[q] != W(0) && f[q] >= 1 && f[q] <= nf - 2;
}

__device__ __forceinline__ void decode(const Geom& g, unsigned t, int dim, int& c, int& i, int& j, int& k) {
  const unsigned N = (unsigned)g.N, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  c = (int)(t / N);
  const unsigned nd = t - (unsigned)c * N;
  const unsigned r = nd / nx;
  i = (int)(nd - r * nx);
  j = dim == 3 ? (int)(r % ny) : (int)r;
  k = dim == 3 ? (int)(r / ny) : 0;
}

// The 1D weights are dyadic (1, 3/4, 3/8, -1/8), so they and their products are
// exact in either precision; the sums run in the vector's precision T.
template <typename T, int DIM>
__device__ __forceinline__ void prolong_body(unsigned bx, const Geom& gc, const Geom& gf, const T* __restrict__ xc,
                                             T* __restrict__ xf, T* __restrict__ xadd) {
  pdl_wait();
  const unsigned t = bx * blockDim.x + threadIdx.x;
  if (t >= (unsigned)(gf.N * DIM)) return;
  int c, i, j, k;
  decode(gf, t, DIM, c, i, j, k);
  if (on_boundary(gf, i, j, k)) { xf[t] = T(0); return; }   // xadd unchanged there
  int mx[3], my[3], mz[3];
  T wx[3], wy[3], wz[3];
  bool ox[3], oy[3], oz[3];
  prolong_taps(i, gc.nn[0], mx, wx, ox);
  prolong_taps(j, gc.nn[1], my, wy, oy);
  if (DIM == 3) prolong_taps(k, gc.nn[2], mz, wz, oz);
  else { mz[0] = mz[1] = mz[2] = 0; wz[0] = T(1); wz[1] = wz[2] = T(0); oz[0] = true; oz[1] = oz[2] = false; }
  const T* xcc = xc + (long long)c * gc.N;
  T acc = T(0);
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 3 : 1); ++cz)
#pragma unroll
    for (int cy = 0; cy < 3; ++cy) {
      const long long row = (long long)gc.nn[0] * ((long long)my[cy] + (long long)gc.nn[1] * mz[cz]);
#pragma unroll
      for (int cx = 0; cx < 3; ++cx) {
        const bool use = ox[cx] && oy[cy] && oz[cz];
        const T v = use ? xcc[row + mx[cx]] : T(0);
        acc += wx[cx] * wy[cy] * wz[cz] * v;
      }
    }
  xf[t] = acc;
  if (xadd) xadd[t] += acc;
}
template <typename T, int DIM>
__global__ void k_prolong(Geom gc, Geom gf, const T* __restrict__ xc, T* __restrict__ xf, T* __restrict__ xadd) {
  prolong_body<T, DIM>(blockIdx.x, gc, gf, xc, xf, xadd);
}

template <typename T, int DIM>
__device__ __forceinline__ void restrict_body(unsigned bx, const Geom& gc, const Geom& gf, const T* __restrict__ rf,
                                              const T* __restrict__ sub, T* __restrict__ rc) {
  pdl_wait();
  const unsigned t = bx * blockDim.x + threadIdx.x;
  if (t >= (unsigned)(gc.N * DIM)) return;
  int c, i, j, k;
  decode(gc, t, DIM, c, i, j, k);
  if (on_boundary(gc, i, j, k)) { rc[t] = T(0); return; }
  int fx[5], fy[5], fz[5];
  T wx[5], wy[5], wz[5];
  bool ox[5], oy[5], oz[5];
  restrict_taps(i, gf.nn[0], fx, wx, ox);
  restrict_taps(j, gf.nn[1], fy, wy, oy);
  if (DIM == 3) restrict_taps(k, gf.nn[2], fz, wz, oz);
  else {
    for (int q = 0; q < 5; ++q) { fz[q] = 0; wz[q] = T(0); oz[q] = false; }
    wz[0] = T(1); oz[0] = true;
  }
  const T* rfc = rf + (long long)c * gf.N;
  const T* sbc = sub ? sub + (long long)c * gf.N : nullptr;
  T acc = T(0);
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 5 : 1); ++cz)
#pragma unroll
    for (int cy = 0; cy < 5; ++cy) {
      const long long row = (long long)gf.nn[0] * ((long long)fy[cy] + (long long)gf.nn[1] * fz[cz]);
      T part = T(0);
#pragma unroll
      for (int cx = 0; cx < 5; ++cx) {
        const bool use = ox[cx] && oy[cy] && oz[cz];
        T v = T(0);
        if (use) v = sbc ? rfc[row + fx[cx]] - sbc[row + fx[cx]] : rfc[row + fx[cx]];
        part += wx[cx] * v;
      }
      acc += wy[cy] * wz[cz] * part;
    }
  rc[t] = acc;
}
template <typename T, int DIM>
__global__ void k_restrict(Geom gc, Geom gf, const T* __restrict__ rf, const T* __restrict__ sub, T* __restrict__ rc) {
  restrict_body<T, DIM>(blockIdx.x, gc, gf, rf, sub, rc);
}

// merged launches (batch.cuh), FP32, 2D and 3D instances together
struct TransferArgs {
  Geom gc, gf;
  const float* in;
  float* out;
  float* aux;
};
__global__ void __launch_bounds__(256) k_prolong_b(const __grid_constant__ BatchTab<TransferArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const TransferArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i];
  if (a.gf.dim == 3) prolong_body<float, 3>(bx, a.gc, a.gf, a.in, a.out, a.aux);
  else prolong_body<float, 2>(bx, a.gc, a.gf, a.in, a.out, a.aux);
}
__global__ void __launch_bounds__(256) k_restrict_b(const __grid_constant__ BatchTab<TransferArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const TransferArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i];
  if (a.gf.dim == 3) restrict_body<float, 3>(bx, a.gc, a.gf, a.in, a.aux, a.out);
  else restrict_body<float, 2>(bx, a.gc, a.gf, a.in, a.aux, a.out);
}

void prolong_std(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf, cudaStream_t s,
                 void* xadd) {
  if (fine.k == 3) {
    qk_prolong(coarse, fine, prec, xc, xf, s, xadd);
    return;
  }
  const long long tot = fine.g.N * fine.g.dim;
  const unsigned b = (unsigned)((tot + 255) / 256);
  if (prec == PREC_F64) {
    if (fine.g.dim == 2)
      launch_pdl(k_prolong<double, 2>, b, 256, 0, s, coarse.g, fine.g, (const double*)xc, (double*)xf, (double*)xadd);
    else launch_pdl(k_prolong<double, 3>, b, 256, 0, s, coarse.g, fine.g, (const double*)xc, (double*)xf, (double*)xadd);
  } else {
    if (fine.g.dim == 2)
      launch_pdl(k_prolong<float, 2>, b, 256, 0, s, coarse.g, fine.g, (const float*)xc, (float*)xf, (float*)xadd);
    else launch_pdl(k_prolong<float, 3>, b, 256, 0, s, coarse.g, fine.g, (const float*)xc, (float*)xf, (float*)xadd);
  }
  count_launch(1);
}

void restrict_std(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc, cudaStream_t s,
                  const void* sub) {
  if (fine.k == 3) {
    qk_restrict(coarse, fine, prec, rf, rc, s, sub);
    return;
  }
  const long long tot = coarse.g.N * coarse.g.dim;
  const unsigned b = (unsigned)((tot + 255) / 256);
  if (prec == PREC_F64) {
    if (fine.g.dim == 2)
      launch_pdl(k_restrict<double, 2>, b, 256, 0, s, coarse.g, fine.g, (const double*)rf, (const double*)sub, (double*)rc);
    else launch_pdl(k_restrict<double, 3>, b, 256, 0, s, coarse.g, fine.g, (const double*)rf, (const double*)sub, (double*)rc);
  } else {
    if (fine.g.dim == 2)
      launch_pdl(k_restrict<float, 2>, b, 256, 0, s, coarse.g, fine.g, (const float*)rf, (const float*)sub, (float*)rc);
    else launch_pdl(k_restrict<float, 3>, b, 256, 0, s, coarse.g, fine.g, (const float*)rf, (const float*)sub, (float*)rc);
  }
  count_launch(1);
}

int batch_prolong(const std::vector<BTransfer>& items, cudaStream_t s) {
  std::vector<TransferArgs> a;
  std::vector<unsigned> nb;
  for (const BTransfer& it : items) {
    a.push_back(TransferArgs{it.coarse->g, it.fine->g, (const float*)it.in, (float*)it.out, (float*)it.aux});
    nb.push_back((unsigned)((it.fine->g.N * it.fine->g.dim + 255) / 256));
  }
  const int n = launch_batch(k_prolong_b, a, nb, 256, 0, s);
  count_launch(n);
  return n;
}

int batch_restrict(const std::vector<BTransfer>& items, cudaStream_t s) {
  std::vector<TransferArgs> a;
  std::vector<unsigned> nb;
  for (const BTransfer& it : items) {
    a.push_back(TransferArgs{it.coarse->g, it.fine->g, (const float*)it.in, (float*)it.out, (float*)it.aux});
    nb.push_back((unsigned)((it.coarse->g.N * it.coarse->g.dim + 255) / 256));
  }
  const int n = launch_batch(k_restrict_b, a, nb, 256, 0, s);
  count_launch(n);
  return n;
}

}  // namespace als
