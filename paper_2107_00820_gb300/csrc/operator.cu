// K1: matrix-free application of the augmented Stokes operators on one level.
//
// One thread per cell evaluates the cell's contribution with the sum-factorised
// kernels of cell.cuh and adds it to the nodal output.  Cells are processed in
// 2^d colours (parity of the cell index per axis): cells of one colour share no
// node, so each launch adds with plain loads and stores, and the fixed colour
// order makes every result bitwise reproducible.  Dirichlet rows carry
// the identity (y_D = x_D) and Dirichlet columns are masked (x_D treated as 0),
// which is the constrained operator of Eq. (augstokessys) in the form Firedrake
// and PETSc use.  B u (Eq. (stokessys)) is cell-local and written directly.
#include "cell.cuh"
#include "level.h"

#include <type_traits>

namespace als {

template <typename T>
struct CellConst {
  T s[3];
  T wdet, inv_m0, inv_m1, gamma;
};

template <typename T>
static CellConst<T> cell_const(const Geom& g, double gamma) {
  CellConst<T> c;
  double vol = 1.0;
  double wdet = 1.0;
  for (int k = 0; k < 3; ++k) {
    c.s[k] = (T)(k < g.dim ? 2.0 / g.h[k] : 0.0);
    if (k < g.dim) { vol *= g.h[k]; wdet *= 0.5 * g.h[k]; }
  }
  c.wdet = (T)wdet;
  c.inv_m0 = (T)(1.0 / vol);
  c.inv_m1 = (T)(3.0 / vol);
  c.gamma = (T)gamma;
  return c;
}

template <typename T, int DIM>
__device__ __forceinline__ void cell_coords(const Geom& g, long long cell, int& cx, int& cy, int& cz) {
  cx = (int)(cell % g.n[0]);
  long long r = cell / g.n[0];
  cy = (int)(r % g.n[1]);
  cz = (DIM == 3) ? (int)(r / g.n[1]) : 0;
}

// cells of one colour: index t -> (step i + bx, step j + by, step k + bz);
// step 2 selects one parity class, step 1 (bits 0) all cells
struct Colour {
  int b[3];      // parity bits
  int m[3];      // cells of this colour per axis
  int step;
  long long count;
};

static Colour all_cells(const Geom& g) {
  Colour c{};
  c.step = 1;
  c.count = g.ncells;
  for (int k = 0; k < 3; ++k) { c.b[k] = 0; c.m[k] = g.n[k]; }
  return c;
}

static Colour make_colour(const Geom& g, int colour) {
  Colour c{};
  c.step = 2;
  c.count = 1;
  for (int k = 0; k < 3; ++k) {
    c.b[k] = (k < g.dim) ? (colour >> k) & 1 : 0;
    c.m[k] = (k < g.dim) ? (g.n[k] - c.b[k] + 1) / 2 : 1;
    c.count *= c.m[k];
  }
  return c;
}

__device__ __forceinline__ bool colour_cell(const Colour& col, long long t, int& cx, int& cy, int& cz) {
  if (t >= col.count) return false;
  const int i = (int)(t % col.m[0]);
  const long long r = t / col.m[0];
  const int j = (int)(r % col.m[1]);
  const int k = (int)(r / col.m[1]);
  cx = col.step * i + col.b[0];
  cy = col.step * j + col.b[1];
  cz = col.step * k + col.b[2];
  return true;
}

template <typename T, int DIM, bool RAW>
__device__ __forceinline__ void load_cell(const Geom& g, const T* __restrict__ x, int cx, int cy, int cz,
                                          T (&u)[DIM][Sz<DIM>::NB]) {
#pragma unroll
  for (int a = 0; a < Sz<DIM>::NB; ++a) {
    const int i = 2 * cx + a % 3, j = 2 * cy + (a / 3) % 3, k = (DIM == 3) ? 2 * cz + a / 9 : 0;
    const bool bnd = !RAW && on_boundary(g, i, j, k);
    const long long nd = node_id(g, i, j, k);
#pragma unroll
    for (int c = 0; c < DIM; ++c) u[c][a] = bnd ? T(0) : x[c * g.N + nd];
  }
}

template <typename T, int DIM, bool RAW>
__device__ __forceinline__ void scatter_cell(const Geom& g, T* __restrict__ y, int cx, int cy, int cz,
                                             const T (&yl)[DIM][Sz<DIM>::NB]) {
#pragma unroll
  for (int a = 0; a < Sz<DIM>::NB; ++a) {
    const int i = 2 * cx + a % 3, j = 2 * cy + (a / 3) % 3, k = (DIM == 3) ? 2 * cz + a / 9 : 0;
    if (!RAW && on_boundary(g, i, j, k)) continue;
    const long long nd = node_id(g, i, j, k);
#pragma unroll
    for (int c = 0; c < DIM; ++c) y[c * g.N + nd] += yl[c][a];
  }
}

template <typename T, int DIM, bool TENSOR, int MODE>
__global__ void __launch_bounds__(128) k_apply(Geom g, Colour col, CellConst<T> cc, const T* __restrict__ x,
                                               T* __restrict__ y, const T* __restrict__ coef,
                                               const T* __restrict__ p_in, T* __restrict__ p_out,
                                               long long vstride) {
  constexpr int NB = Sz<DIM>::NB, NPR = Sz<DIM>::NPR;
  constexpr bool RAW = (MODE & OP_RAW) != 0;
  x += blockIdx.y * vstride;
  y += blockIdx.y * vstride;
  constexpr int NCQ = TENSOR ? Sz<DIM>::NC : 1;
  constexpr bool NEED_U = (MODE & (OP_VISC | OP_AL | OP_B)) != 0;
  constexpr bool NEED_FLUX = (MODE & (OP_VISC | OP_AL | OP_BT)) != 0;
  int cx, cy, cz;
  if (!colour_cell(col, (long long)blockIdx.x * blockDim.x + threadIdx.x, cx, cy, cz)) return;
  const long long cell = (long long)cx + (long long)g.n[0] * ((long long)cy + (long long)g.n[1] * cz);
  T u[DIM][NB];
  if constexpr (NEED_U) load_cell<T, DIM, RAW>(g, x, cx, cy, cz, u);
  else {
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int a = 0; a < NB; ++a) u[c][a] = T(0);
  }
  T pi[NPR];
#pragma unroll
  for (int p = 0; p < NPR; ++p) pi[p] = T(0);
  if constexpr ((MODE & (OP_AL | OP_B)) != 0) {
    T m[NPR];
    div_moments<T, DIM>(u, cc.s, cc.wdet, m);
    if constexpr ((MODE & OP_B) != 0) {
#pragma unroll
      for (int p = 0; p < NPR; ++p) p_out[cell * NPR + p] = -m[p];
    }
    if constexpr ((MODE & OP_AL) != 0) {
#pragma unroll
      for (int p = 0; p < NPR; ++p) pi[p] += cc.gamma * m[p] * (p == 0 ? cc.inv_m0 : cc.inv_m1);
    }
  }
  if constexpr ((MODE & OP_BT) != 0) {
#pragma unroll
    for (int p = 0; p < NPR; ++p) pi[p] -= p_in[cell * NPR + p];
  }
  if constexpr (NEED_FLUX) {
    T yl[DIM][NB];
    cell_flux_apply<T, DIM, TENSOR, (MODE & OP_VISC) != 0>(u, coef + cell * NB * NCQ, cc.s, cc.wdet, pi, yl);
    scatter_cell<T, DIM, RAW>(g, y, cx, cy, cz, yl);
  }
}

// y_D = x_D (identity rows) when keep_bnd, else 0; interior rows zeroed.
template <typename T>
__global__ void k_init_out(Geom g, const T* __restrict__ x, T* __restrict__ y, int keep_bnd, long long vstride) {
  x += blockIdx.y * vstride;
  y += blockIdx.y * vstride;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = g.N * g.dim;
  if (t >= total) return;
  const long long nd = t % g.N;
  const int i = (int)(nd % g.nn[0]);
  const long long r = nd / g.nn[0];
  const int j = (int)(r % g.nn[1]);
  const int k = (int)(r / g.nn[1]);
  const bool bnd = on_boundary(g, i, j, k);
  y[t] = (bnd && keep_bnd) ? x[t] : T(0);
}

template <typename T, int DIM, bool TENSOR, int MODE>
static void launch_apply(const LevelDev& L, double gamma, const void* x, void* y, const void* p_in,
                         void* p_out, int nvec, long long vstride, cudaStream_t s) {
  const Geom& g = L.g;
  constexpr bool NEED_FLUX = (MODE & (OP_VISC | OP_AL | OP_BT)) != 0;
  for (int v0 = 0; v0 < nvec; v0 += 65535) {
    const int nv = nvec - v0 < 65535 ? nvec - v0 : 65535;
    const T* xv = (const T*)x + v0 * vstride;
    T* yv = (T*)y + v0 * vstride;
    if (NEED_FLUX) {
      const long long tot = g.N * g.dim;
      dim3 grid((unsigned)((tot + 255) / 256), nv);
      k_init_out<T><<<grid, 256, 0, s>>>(g, xv, yv, ((MODE & OP_VISC) && !(MODE & OP_RAW)) ? 1 : 0, vstride);
    }
    const T* coef = nullptr;
    if constexpr (std::is_same<T, double>::value) coef = L.coef64; else coef = L.coef32;
    const int ncol = NEED_FLUX ? (1 << DIM) : 1;   // B u alone is cell-local: one launch
    for (int colour = 0; colour < ncol; ++colour) {
      const Colour col = NEED_FLUX ? make_colour(g, colour) : all_cells(g);
      dim3 grid((unsigned)((col.count + 127) / 128), nv);
      k_apply<T, DIM, TENSOR, MODE><<<grid, 128, 0, s>>>(g, col, cell_const<T>(g, gamma), xv, yv, coef,
                                                         (const T*)p_in, (T*)p_out, vstride);
    }
    count_launch((NEED_FLUX ? 1 : 0) + ncol);
  }
}

template <typename T, int DIM, bool TENSOR>
static void dispatch_mode(const LevelDev& L, int mode, double gamma, const void* x, void* y,
                          const void* p_in, void* p_out, int nvec, long long vstride, cudaStream_t s) {
  switch (mode) {
    case OP_VISC | OP_AL:
      launch_apply<T, DIM, TENSOR, OP_VISC | OP_AL>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
    case OP_AL: launch_apply<T, DIM, TENSOR, OP_AL>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
    default:
      if constexpr (std::is_same<T, double>::value) {
        switch (mode) {
          case OP_VISC | OP_AL | OP_BT | OP_B:
            launch_apply<T, DIM, TENSOR, OP_VISC | OP_AL | OP_BT | OP_B>(L, gamma, x, y, p_in, p_out, nvec, vstride, s);
            break;
          case OP_B: launch_apply<T, DIM, TENSOR, OP_B>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
          case OP_BT: launch_apply<T, DIM, TENSOR, OP_BT>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
          case OP_VISC | OP_AL | OP_RAW:
            launch_apply<T, DIM, TENSOR, OP_VISC | OP_AL | OP_RAW>(L, gamma, x, y, p_in, p_out, nvec, vstride, s);
            break;
          case OP_B | OP_RAW:
            launch_apply<T, DIM, TENSOR, OP_B | OP_RAW>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
          default: break;
        }
      }
      break;
  }
}

static void op_dispatch(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y,
                        const void* p_in, void* p_out, int nvec, long long vstride, cudaStream_t s) {
  if (prec == PREC_F64) {
    if (L.g.dim == 2) {
      if (L.tensor) dispatch_mode<double, 2, true>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
      else dispatch_mode<double, 2, false>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
    } else {
      if (L.tensor) dispatch_mode<double, 3, true>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
      else dispatch_mode<double, 3, false>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
    }
  } else {
    if (L.g.dim == 2) {
      if (L.tensor) dispatch_mode<float, 2, true>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
      else dispatch_mode<float, 2, false>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
    } else {
      if (L.tensor) dispatch_mode<float, 3, true>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
      else dispatch_mode<float, 3, false>(L, mode, gamma, x, y, p_in, p_out, nvec, vstride, s);
    }
  }
}

void op_apply(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y,
              const void* p_in, void* p_out, cudaStream_t s) {
  op_dispatch(L, prec, mode, gamma, x, y, p_in, p_out, 1, 0, s);
}

// Several independent FP64 applies of A_gamma (used to form the coarse matrix
// column by column from unit vectors): vector v at X + v*stride.
void op_apply_multi(const LevelDev& L, double gamma, const double* X, double* Y, int nvec,
                    long long stride, cudaStream_t s) {
  op_dispatch(L, PREC_F64, OP_VISC | OP_AL, gamma, X, Y, nullptr, nullptr, nvec, stride, s);
}

// F_(c,a) = sum_q |J| w_q f_c(x_q) phi_a(x_q): the load vector of the body force.
template <int DIM>
__global__ void k_load(Geom g, Colour col, double wdet, const double* __restrict__ f, double* __restrict__ F) {
  constexpr int NB = Sz<DIM>::NB;
  int cx, cy, cz;
  if (!colour_cell(col, (long long)blockIdx.x * blockDim.x + threadIdx.x, cx, cy, cz)) return;
  const long long cell = (long long)cx + (long long)g.n[0] * ((long long)cy + (long long)g.n[1] * cz);
  double loc[DIM][NB];
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int a = 0; a < NB; ++a) loc[c][a] = 0.0;
  for (int q = 0; q < NB; ++q) {
    const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
    double w = wdet * Ref<double>::W(qx) * Ref<double>::W(qy) * (DIM == 3 ? Ref<double>::W(qz) : 1.0);
    double fq[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) fq[c] = f[(cell * NB + q) * DIM + c] * w;
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      const int ax = a % 3, ay = (a / 3) % 3, az = a / 9;
      const double phi = Ref<double>::B(qx, ax) * Ref<double>::B(qy, ay) * (DIM == 3 ? Ref<double>::B(qz, az) : 1.0);
#pragma unroll
      for (int c = 0; c < DIM; ++c) loc[c][a] += fq[c] * phi;
    }
  }
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    const int i = 2 * cx + a % 3, j = 2 * cy + (a / 3) % 3, k = (DIM == 3) ? 2 * cz + a / 9 : 0;
    const long long nd = node_id(g, i, j, k);
#pragma unroll
    for (int c = 0; c < DIM; ++c) F[c * g.N + nd] += loc[c][a];
  }
}

void op_load_vector(const LevelDev& L, const double* f_qp, double* F, cudaStream_t s) {
  const Geom& g = L.g;
  double wdet = 1.0;
  for (int k = 0; k < g.dim; ++k) wdet *= 0.5 * g.h[k];
  cudaMemsetAsync(F, 0, sizeof(double) * g.N * g.dim, s);
  for (int colour = 0; colour < (1 << g.dim); ++colour) {
    const Colour col = make_colour(g, colour);
    const unsigned blocks = (unsigned)((col.count + 127) / 128);
    if (g.dim == 2) k_load<2><<<blocks, 128, 0, s>>>(g, col, wdet, f_qp, F);
    else k_load<3><<<blocks, 128, 0, s>>>(g, col, wdet, f_qp, F);
  }
  count_launch(1 << g.dim);
}

}  // namespace als
