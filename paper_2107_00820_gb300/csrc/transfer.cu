// K5: standard Q2 prolongation P_H and its transpose (Sec. 5.2).
//
// V_H is a subspace of V_h, so P_H is nested interpolation: a fine node at a
// coarse node takes its value; a fine node at a quarter point of a coarse cell
// takes the coarse quadratic there, 1D weights (3/8, 3/4, -1/8) at 1/4 and
// (-1/8, 3/4, 3/8) at 3/4, tensorised over the axes.  Dirichlet rows (fine
// boundary) and columns (coarse boundary) are zero.  Both directions are
// gathers (one thread per output value), so they need no atomics.
#include "level.h"

namespace als {

template <int DIM>
__device__ __forceinline__ void node_ijk(const Geom& g, long long nd, int& i, int& j, int& k) {
  i = (int)(nd % g.nn[0]);
  const long long r = nd / g.nn[0];
  j = (int)(r % g.nn[1]);
  k = (DIM == 3) ? (int)(r / g.nn[1]) : 0;
}

// fine node f (1D): coarse nodes and weights of the interpolation
__device__ __forceinline__ int prolong_weights_1d(int f, int* m, double* w) {
  if ((f & 1) == 0) { m[0] = f >> 1; w[0] = 1.0; return 1; }
  const int c = f >> 2;           // coarse cell
  const bool first = (f & 3) == 1;
  m[0] = 2 * c; m[1] = 2 * c + 1; m[2] = 2 * c + 2;
  w[0] = first ? 0.375 : -0.125; w[1] = 0.75; w[2] = first ? -0.125 : 0.375;
  return 3;
}

// coarse node m (1D): fine nodes and weights of the transpose (nf = fine nodes per axis)
__device__ __forceinline__ int restrict_weights_1d(int m, int nf, int* f, double* w) {
  int cnt = 0;
  auto add = [&](int ff, double ww) { if (ff >= 0 && ff < nf) { f[cnt] = ff; w[cnt] = ww; ++cnt; } };
  add(2 * m, 1.0);
  if (m & 1) { add(2 * m - 1, 0.75); add(2 * m + 1, 0.75); }
  else { add(2 * m - 1, 0.375); add(2 * m + 1, 0.375); add(2 * m - 3, -0.125); add(2 * m + 3, -0.125); }
  return cnt;
}

template <typename T, int DIM>
__global__ void k_prolong(Geom gc, Geom gf, const T* __restrict__ xc, T* __restrict__ xf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gf.N * DIM) return;
  const int c = (int)(t / gf.N);
  int i, j, k;
  node_ijk<DIM>(gf, t % gf.N, i, j, k);
  if (on_boundary(gf, i, j, k)) { xf[t] = T(0); return; }
  int mx[3], my[3], mz[3] = {0, 0, 0};
  double wx[3], wy[3], wz[3] = {1.0, 0.0, 0.0};
  const int nx = prolong_weights_1d(i, mx, wx), ny = prolong_weights_1d(j, my, wy);
  const int nz = DIM == 3 ? prolong_weights_1d(k, mz, wz) : 1;
  double acc = 0.0;
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx) {
        if (on_boundary(gc, mx[cx], my[cy], mz[cz])) continue;
        acc += wx[cx] * wy[cy] * wz[cz] * (double)xc[c * gc.N + node_id(gc, mx[cx], my[cy], mz[cz])];
      }
  xf[t] = (T)acc;
}

template <typename T, int DIM>
__global__ void k_restrict(Geom gc, Geom gf, const T* __restrict__ rf, T* __restrict__ rc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.N * DIM) return;
  const int c = (int)(t / gc.N);
  int i, j, k;
  node_ijk<DIM>(gc, t % gc.N, i, j, k);
  if (on_boundary(gc, i, j, k)) { rc[t] = T(0); return; }
  int fx[5], fy[5], fz[5] = {0, 0, 0, 0, 0};
  double wx[5], wy[5], wz[5] = {1.0, 0, 0, 0, 0};
  const int nx = restrict_weights_1d(i, gf.nn[0], fx, wx), ny = restrict_weights_1d(j, gf.nn[1], fy, wy);
  const int nz = DIM == 3 ? restrict_weights_1d(k, gf.nn[2], fz, wz) : 1;
  double acc = 0.0;
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx) {
        if (on_boundary(gf, fx[cx], fy[cy], fz[cz])) continue;
        acc += wx[cx] * wy[cy] * wz[cz] * (double)rf[c * gf.N + node_id(gf, fx[cx], fy[cy], fz[cz])];
      }
  rc[t] = (T)acc;
}

void prolong_std(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf, cudaStream_t s) {
  const long long tot = fine.g.N * fine.g.dim;
  const unsigned b = (unsigned)((tot + 255) / 256);
  if (prec == PREC_F64) {
    if (fine.g.dim == 2) k_prolong<double, 2><<<b, 256, 0, s>>>(coarse.g, fine.g, (const double*)xc, (double*)xf);
    else k_prolong<double, 3><<<b, 256, 0, s>>>(coarse.g, fine.g, (const double*)xc, (double*)xf);
  } else {
    if (fine.g.dim == 2) k_prolong<float, 2><<<b, 256, 0, s>>>(coarse.g, fine.g, (const float*)xc, (float*)xf);
    else k_prolong<float, 3><<<b, 256, 0, s>>>(coarse.g, fine.g, (const float*)xc, (float*)xf);
  }
  count_launch(1);
}

void restrict_std(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc, cudaStream_t s) {
  const long long tot = coarse.g.N * coarse.g.dim;
  const unsigned b = (unsigned)((tot + 255) / 256);
  if (prec == PREC_F64) {
    if (fine.g.dim == 2) k_restrict<double, 2><<<b, 256, 0, s>>>(coarse.g, fine.g, (const double*)rf, (double*)rc);
    else k_restrict<double, 3><<<b, 256, 0, s>>>(coarse.g, fine.g, (const double*)rf, (double*)rc);
  } else {
    if (fine.g.dim == 2) k_restrict<float, 2><<<b, 256, 0, s>>>(coarse.g, fine.g, (const float*)rf, (float*)rc);
    else k_restrict<float, 3><<<b, 256, 0, s>>>(coarse.g, fine.g, (const float*)rf, (float*)rc);
  }
  count_launch(1);
}

}  // namespace als
