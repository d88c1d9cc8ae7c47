// K1: matrix-free application of the augmented Stokes operators on one level.
//
// One warp per cell (three in 2D) evaluates the cell's contribution with sum
// factorisation.  The nodal sum is formed without atomics, in a fixed order so
// every result is bitwise reproducible: normally all cells write their local
// outputs to a per-cell buffer and one gather kernel sums the <= 2^d values of
// each node (two launches per apply); batched applies (many vectors at once)
// instead run the cells in 2^d colours (parity of the cell index per axis) whose
// cells share no node and add into y directly.  Dirichlet rows carry
// the identity (y_D = x_D) and Dirichlet columns are masked (x_D treated as 0),
// which is the constrained operator of Eq. (augstokessys) in the form Firedrake
// and PETSc use.  B u (Eq. (stokessys)) is cell-local and written directly.
#include "batch.cuh"
#include "cell.cuh"
#include "level.h"
#include "reduce.cuh"
#include "pdl.cuh"

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

// 32-bit arithmetic: cell counts stay below 2^31 (checked when a context is created)
__device__ __forceinline__ bool colour_cell(const Colour& col, long long t, int& cx, int& cy, int& cz) {
  if (t >= col.count) return false;
  const unsigned tu = (unsigned)t, m0 = (unsigned)col.m[0], m1 = (unsigned)col.m[1];
  const unsigned r = tu / m0;
  const int i = (int)(tu - r * m0);
  const unsigned k = r / m1;
  const int j = (int)(r - k * m1);
  cx = col.step * i + col.b[0];
  cy = col.step * j + col.b[1];
  cz = col.step * k + col.b[2];
  return true;
}

// One warp evaluates one cell (3D: 27 lanes = 27 nodes = 27 Gauss points) or
// three cells (2D: 9 lanes each).  The three 1D contractions of the sum
// factorisation run lane-parallel through shared memory, the divergence
// moments are a warp (3D) or lane-group (2D) reduction, and the isotropic AL /
// pressure part of the stress is formed at every point before the transposed
// contractions take the fluxes back to the nodes.
template <typename T, int DIM, bool TENSOR, int MODE, bool STAGED>
__device__ __forceinline__ void apply_body(unsigned bx, const Geom& g, const Colour& col, const CellConst<T>& cc,
                                           const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ coef,
                                           const T* __restrict__ p_in, T* __restrict__ p_out, long long vstride,
                                           T* __restrict__ ebuf, const T* __restrict__ winv) {
  constexpr int NB = Sz<DIM>::NB, NPR = Sz<DIM>::NPR;
  constexpr int CPW = DIM == 2 ? 3 : 1;        // cells per warp
  constexpr int NCQ = TENSOR ? Sz<DIM>::NC : 1;
  constexpr bool RAW = (MODE & OP_RAW) != 0;
  constexpr bool VISC = (MODE & OP_VISC) != 0;
  constexpr bool NEED_U = (MODE & (OP_VISC | OP_AL | OP_B)) != 0;
  constexpr bool NEED_FLUX = (MODE & (OP_VISC | OP_AL | OP_BT)) != 0;
  __shared__ T sh[8][2][9][27];
  x += blockIdx.y * vstride;
  y += blockIdx.y * vstride;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / NB < CPW ? lane / NB : 0;
  const bool lane_ok = lane < CPW * NB;
  const int l = lane_ok ? lane - grp * NB : 0;
  const int base = grp * NB;
  T (*SA)[27] = sh[w][0];
  T (*SB)[27] = sh[w][1];
  const long long t = ((long long)bx * (blockDim.x >> 5) + w) * CPW + grp;
  int cx = 0, cy = 0, cz = 0;
  const bool act = lane_ok && colour_cell(col, t, cx, cy, cz);
  const long long cell = (long long)(unsigned)(cx + g.n[0] * (cy + g.n[1] * cz));
  const int i0 = l % 3, i1 = (l / 3) % 3, i2 = DIM == 3 ? l / 9 : 0;
  const int ni = 2 * cx + i0, nj = 2 * cy + i1, nk = DIM == 3 ? 2 * cz + i2 : 0;
  const long long nd = (long long)(unsigned)(ni + g.nn[0] * (nj + g.nn[1] * nk));
  const bool bnd = on_boundary(g, ni, nj, nk);

  T grad[DIM][DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int k = 0; k < DIM; ++k) grad[c][k] = T(0);
  pdl_wait();

  if constexpr (NEED_U) {
    // stage 1: nodal values (Dirichlet columns masked unless RAW)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const T v = (act && (RAW || !bnd)) ? x[c * g.N + nd] : T(0);
      if (lane_ok) SA[c][base + l] = v;
    }
    __syncwarp();
    if constexpr (DIM == 3) {
      // stage 2 (x): lane = (qx, ay, az): B_x u, D_x u
      if (lane_ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T t0 = T(0), t1 = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T v = SA[c][a + 3 * i1 + 9 * i2];
            t0 += Ref<T>::B(i0, a) * v;
            t1 += Ref<T>::D(i0, a) * v;
          }
          SB[c][l] = t0;
          SB[3 + c][l] = t1;
        }
      }
      __syncwarp();
      // stage 3 (y): lane = (qx, qy, az): B_x B_y u, B_x D_y u, D_x B_y u
      if (lane_ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const T v0 = SB[c][i0 + 3 * b + 9 * i2], v1 = SB[3 + c][i0 + 3 * b + 9 * i2];
            a0 += Ref<T>::B(i1, b) * v0;
            a1 += Ref<T>::D(i1, b) * v0;
            a2 += Ref<T>::B(i1, b) * v1;
          }
          SA[c][l] = a0;
          SA[3 + c][l] = a1;
          SA[6 + c][l] = a2;
        }
      }
      __syncwarp();
      // stage 4 (z): lane = (qx, qy, qz): the gradient at this point
      if (lane_ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int idx = i0 + 3 * i1 + 9 * k;
            gx += Ref<T>::B(i2, k) * SA[6 + c][idx];
            gy += Ref<T>::B(i2, k) * SA[3 + c][idx];
            gz += Ref<T>::D(i2, k) * SA[c][idx];
          }
          grad[c][0] = gx * cc.s[0];
          grad[c][1] = gy * cc.s[1];
          grad[c][2] = gz * cc.s[2];
        }
      }
    } else {
      // stage 2 (x): lane = (qx, ay): B_x u, D_x u
      if (lane_ok) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          T t0 = T(0), t1 = T(0);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T v = SA[c][base + a + 3 * i1];
            t0 += Ref<T>::B(i0, a) * v;
            t1 += Ref<T>::D(i0, a) * v;
          }
          SB[c][base + l] = t0;
          SB[2 + c][base + l] = t1;
        }
      }
      __syncwarp();
      // stage 3 (y): lane = (qx, qy)
      if (lane_ok) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          T gx = T(0), gy = T(0);
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            gx += Ref<T>::B(i1, b) * SB[2 + c][base + i0 + 3 * b];
            gy += Ref<T>::D(i1, b) * SB[c][base + i0 + 3 * b];
          }
          grad[c][0] = gx * cc.s[0];
          grad[c][1] = gy * cc.s[1];
        }
      }
    }
  }

  // point weight, pressure basis at this point
  const T wq = cc.wdet * Ref<T>::W(i0) * Ref<T>::W(i1) * (DIM == 3 ? Ref<T>::W(i2) : T(1));
  T psi[NPR];
  psi[0] = T(1);
  psi[1] = Ref<T>::G(i0);
  psi[2] = Ref<T>::G(i1);
  if constexpr (DIM == 3) psi[3] = Ref<T>::G(i2);

  // divergence moments m_p = (psi_p, div u)_K
  T m[NPR];
#pragma unroll
  for (int p = 0; p < NPR; ++p) m[p] = T(0);
  if constexpr ((MODE & (OP_AL | OP_B)) != 0) {
    T dv = T(0);
#pragma unroll
    for (int c = 0; c < DIM; ++c) dv += grad[c][c];
    dv = lane_ok ? wq * dv : T(0);
    if constexpr (DIM == 3) {
#pragma unroll
      for (int p = 0; p < NPR; ++p) {
        T v = dv * psi[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        m[p] = v;
      }
    } else {
      __syncwarp();
      if (lane_ok) {
#pragma unroll
        for (int p = 0; p < NPR; ++p) SB[p][base + l] = dv * psi[p];
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < NPR; ++p) {
        T v = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) v += SB[p][base + q];
        m[p] = v;
      }
    }
    if constexpr ((MODE & OP_B) != 0) {
      if (act && l < NPR) p_out[cell * NPR + l] = -m[l];
    }
  }
  if constexpr (NEED_FLUX) {
  // isotropic part of the stress: gamma Pi div u - p_h
  T pi[NPR];
#pragma unroll
  for (int p = 0; p < NPR; ++p) {
    pi[p] = T(0);
    if constexpr ((MODE & OP_AL) != 0) {
      if (winv) {   // W = M_p(1/mu): per-cell (d+1)^2 block of W^-1
        T acc = T(0);
        if (act) {
#pragma unroll
          for (int q = 0; q < NPR; ++q) acc += winv[(cell * NPR + p) * NPR + q] * m[q];
        }
        pi[p] += cc.gamma * acc;
      } else {      // W = M_p = |K| diag(1, 1/3, ..)
        pi[p] += cc.gamma * m[p] * (p == 0 ? cc.inv_m0 : cc.inv_m1);
      }
    }
    if constexpr ((MODE & OP_BT) != 0) pi[p] -= act ? p_in[cell * NPR + p] : T(0);
  }
  T iso = T(0);
#pragma unroll
  for (int p = 0; p < NPR; ++p) iso += pi[p] * psi[p];
  T sg[DIM][DIM];
  if constexpr (VISC) {
    if (act) stress<T, DIM, TENSOR>(coef + (cell * NB + l) * NCQ, grad, iso, sg);
    else {
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int k = 0; k < DIM; ++k) sg[c][k] = T(0);
    }
  } else {
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int k = 0; k < DIM; ++k) sg[c][k] = (c == k) ? iso : T(0);
  }
  __syncwarp();
  // fluxes F[c][k] = |J| w_q sigma_ck (2/h_k)
  if (lane_ok) {
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int k = 0; k < DIM; ++k) SA[DIM * c + k][base + l] = wq * sg[c][k] * cc.s[k];
  }
  __syncwarp();
  T yl[DIM];
  if constexpr (DIM == 3) {
    // stage 5 (z^T): lane = (qx, qy, az)
    if (lane_ok) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T ge = T(0), gb = T(0), ga = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int idx = i0 + 3 * i1 + 9 * q;
          ge += Ref<T>::B(q, i2) * SA[3 * c + 0][idx];
          gb += Ref<T>::B(q, i2) * SA[3 * c + 1][idx];
          ga += Ref<T>::D(q, i2) * SA[3 * c + 2][idx];
        }
        SB[c][l] = ge;
        SB[3 + c][l] = gb;
        SB[6 + c][l] = ga;
      }
    }
    __syncwarp();
    // stage 6 (y^T): lane = (qx, ay, az)
    if (lane_ok) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T p0 = T(0), p1 = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int idx = i0 + 3 * q + 9 * i2;
          p0 += Ref<T>::B(q, i1) * SB[6 + c][idx] + Ref<T>::D(q, i1) * SB[3 + c][idx];
          p1 += Ref<T>::B(q, i1) * SB[c][idx];
        }
        SA[c][l] = p0;
        SA[3 + c][l] = p1;
      }
    }
    __syncwarp();
    // stage 7 (x^T): lane = (ax, ay, az)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int idx = q + 3 * i1 + 9 * i2;
        v += Ref<T>::B(q, i0) * SA[c][idx] + Ref<T>::D(q, i0) * SA[3 + c][idx];
      }
      yl[c] = v;
    }
  } else {
    // stage 5 (y^T): lane = (qx, ay)
    if (lane_ok) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T p0 = T(0), p1 = T(0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int idx = base + i0 + 3 * q;
          p0 += Ref<T>::D(q, i1) * SA[2 * c + 1][idx];
          p1 += Ref<T>::B(q, i1) * SA[2 * c + 0][idx];
        }
        SB[c][base + l] = p0;
        SB[2 + c][base + l] = p1;
      }
    }
    __syncwarp();
    // stage 6 (x^T): lane = (ax, ay)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int idx = base + q + 3 * i1;
        v += Ref<T>::B(q, i0) * SB[c][idx] + Ref<T>::D(q, i0) * SB[2 + c][idx];
      }
      yl[c] = v;
    }
  }
  if constexpr (STAGED) {
    // staged outputs in the row layout (stage_row), summed per node by the gather in a fixed order
    if (act) {
#pragma unroll
      for (int c = 0; c < DIM; ++c)
        ebuf[(long long)stage_row(g, c, i1, i2, cy, cz) * (3 * g.n[0]) + 3 * cx + i0] = yl[c];
    }
  } else {
    if (act && (RAW || !bnd)) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) y[c * g.N + nd] += yl[c];
    }
  }
  }  // NEED_FLUX
  pdl_trigger();
}
template <typename T, int DIM, bool TENSOR, int MODE, bool STAGED>
__global__ void __launch_bounds__(256) k_apply(Geom g, Colour col, CellConst<T> cc, const T* __restrict__ x,
                                               T* __restrict__ y, const T* __restrict__ coef,
                                               const T* __restrict__ p_in, T* __restrict__ p_out,
                                               long long vstride, T* __restrict__ ebuf,
                                               const T* __restrict__ winv) {
  apply_body<T, DIM, TENSOR, MODE, STAGED>(blockIdx.x, g, col, cc, x, y, coef, p_in, p_out, vstride, ebuf, winv);
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

// (A x) along a row of global nodes: one thread sums GX = 4 consecutive nodes
// x = 4j .. 4j+3 of row (c, y, z) from the staged outputs (row layout, see
// stage_row).  Per (y, z) tap pair the four nodes read the six contiguous
// columns 6j-1 .. 6j+4; a column exists iff it lies in [0, 3 n0).  The taps are
// added in a fixed order (z tap, y tap, then the x pair), so results are
// reproducible.  Dirichlet rows: x_D (keep_bnd) or 0, unless raw.
template <typename T, int DIM>
__device__ __forceinline__ void gather_chunk(const Geom& g, const T* __restrict__ ebuf, const T* __restrict__ x,
                                             const RowChunk& rc, int keep_bnd, int raw, T (&out)[GX]) {
  const int nn0 = g.nn[0];
  const bool row_bnd = rc.y == 0 || rc.y == g.nn[1] - 1 || (DIM == 3 && (rc.z == 0 || rc.z == g.nn[2] - 1));
  if (!raw && row_bnd) {
#pragma unroll
    for (int q = 0; q < GX; ++q) {
      const int xi = GX * rc.j + q;
      out[q] = (keep_bnd && xi < nn0) ? x[rc.t0 + q] : T(0);
    }
    return;
  }
  // y and z taps: (cell, local index, exists)
  int cyv[2], lyv[2], czv[2], lzv[2];
  bool oky[2], okz[2];
  {
    const int yy = rc.y;
    if (yy & 1) { cyv[0] = yy >> 1; lyv[0] = 1; oky[0] = true; cyv[1] = 0; lyv[1] = 0; oky[1] = false; }
    else { cyv[0] = (yy >> 1) - 1; lyv[0] = 2; oky[0] = yy > 0; cyv[1] = yy >> 1; lyv[1] = 0; oky[1] = yy < 2 * g.n[1]; }
    const int zz = DIM == 3 ? rc.z : 1;
    const int n2 = DIM == 3 ? g.n[2] : 1;
    if (zz & 1) { czv[0] = zz >> 1; lzv[0] = 1; okz[0] = true; czv[1] = 0; lzv[1] = 0; okz[1] = false; }
    else { czv[0] = (zz >> 1) - 1; lzv[0] = 2; okz[0] = zz > 0; czv[1] = zz >> 1; lzv[1] = 0; okz[1] = zz < 2 * n2; }
    if (DIM == 2) { czv[0] = 0; lzv[0] = 0; }
  }
  const int ncol = 3 * g.n[0];
  const int p0 = 6 * rc.j - 1;
  T acc[GX];
#pragma unroll
  for (int q = 0; q < GX; ++q) acc[q] = T(0);
#pragma unroll
  for (int tz = 0; tz < (DIM == 3 ? 2 : 1); ++tz)
#pragma unroll
    for (int ty = 0; ty < 2; ++ty) {
      if (!(oky[ty] && (DIM == 2 || okz[tz]))) continue;
      const T* rowp = ebuf + (long long)stage_row(g, rc.c, lyv[ty], lzv[tz], cyv[ty], czv[tz]) * ncol;
      T v[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const int p = p0 + k;
        v[k] = (p >= 0 && p < ncol) ? rowp[p] : T(0);
      }
      acc[0] += v[0] + v[1];
      acc[1] += v[2];
      acc[2] += v[3] + v[4];
      acc[3] += v[5];
    }
#pragma unroll
  for (int q = 0; q < GX; ++q) {
    const int xi = GX * rc.j + q;
    if (!raw && (xi == 0 || xi == nn0 - 1)) acc[q] = (keep_bnd && xi < nn0) ? x[rc.t0 + q] : T(0);
    out[q] = acc[q];
  }
}

template <typename T, int DIM>
__device__ __forceinline__ void gather_cells_body(unsigned bx, const Geom& g, const T* __restrict__ ebuf,
                                                  const T* __restrict__ x, T* __restrict__ y, int keep_bnd, int raw) {
  pdl_wait();
  RowChunk rc;
  if (!row_chunk(g, DIM, bx * blockDim.x + threadIdx.x, rc)) return;
  T out[GX];
  gather_chunk<T, DIM>(g, ebuf, x, rc, keep_bnd, raw, out);
#pragma unroll
  for (int q = 0; q < GX; ++q)
    if (GX * rc.j + q < g.nn[0]) y[rc.t0 + q] = out[q];
}
template <typename T, int DIM>
__global__ void k_gather_cells(Geom g, const T* __restrict__ ebuf, const T* __restrict__ x, T* __restrict__ y,
                               int keep_bnd, int raw) {
  gather_cells_body<T, DIM>(blockIdx.x, g, ebuf, x, y, keep_bnd, raw);
}

static unsigned gather_threads(const Geom& g) {
  return (unsigned)(g.dim * g.nn[1] * g.nn[2] * ((g.nn[0] + GX - 1) / GX));
}

// Gather fused with the reduction that consumes the result:
//   y = b + sigma A x (b NULL: y = sigma A x);  out[j] = (V_j . y) / hn[j], j < k;
//   start: |y|^2 starts a GMRES cycle.  Fixed grid and order: reproducible.
// All sums run in T (in FP32 the GMRES state is float too, see GmresView).
template <typename T, int DIM>
__device__ __forceinline__ void gather_epi_body(unsigned bx, unsigned nb, const Geom& g, const T* __restrict__ ebuf,
                                                const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ b,
                                                double sigma, int k, const T* __restrict__ V, long long ld,
                                                T* __restrict__ out, int start, GmresDev sd,
                                                double* __restrict__ partial) {
  __shared__ T nrm2_s[1];
  const GmresView<T> st = gmres_view<T>(sd);
  T* rows = reinterpret_cast<T*>(partial + 1);
  const int kk = start ? 1 : k;
  T acc[KMAXB];
#pragma unroll
  for (int j = 0; j < KMAXB; ++j) acc[j] = T(0);
  RowChunk rc;
  const bool have = row_chunk(g, DIM, bx * blockDim.x + threadIdx.x, rc);
  // The basis columns come from earlier kernels of the chain, which completed before
  // this launch began (every kernel waits on its predecessor before it lets its
  // successor start): they are read through L2 while the preceding kernel finishes.
  T vp[GX][KMAXB];
#pragma unroll
  for (int q = 0; q < GX; ++q)
#pragma unroll
    for (int jj = 0; jj < KMAXB; ++jj)
      vp[q][jj] = (!start && have && jj < k && GX * rc.j + q < g.nn[0]) ? __ldcg(V + (long long)jj * ld + rc.t0 + q)
                                                                         : T(0);
  pdl_wait();
  if (have) {
    T ax[GX];
    gather_chunk<T, DIM>(g, ebuf, x, rc, 1, 0, ax);
#pragma unroll
    for (int q = 0; q < GX; ++q) {
      if (GX * rc.j + q >= g.nn[0]) break;
      const long long t = rc.t0 + q;
      const T v = (b ? b[t] : T(0)) + (T)sigma * ax[q];
      y[t] = v;
      if (start) {
        acc[0] += v * v;
      } else {
#pragma unroll
        for (int jj = 0; jj < KMAXB; ++jj)
          if (jj < k) acc[jj] += vp[q][jj] * v;
      }
    }
  }
  pdl_trigger();
  block_partials<T, T>(acc, kk, rows + (long long)bx * kk);
  if (last_block(partial, nb)) {
    if (start) {
      finish_sums_n<T>(partial, 1, nrm2_s, nullptr, (int)nb);
      if (threadIdx.x == 0) gmres_start(st, nrm2_s[0]);
    } else {
      finish_sums_n<T>(partial, k, out, st.hn, (int)nb);
    }
  }
}
template <typename T, int DIM>
__global__ void __launch_bounds__(RED_THREADS) k_gather_epi(Geom g, const T* __restrict__ ebuf,
                                                            const T* __restrict__ x, T* __restrict__ y,
                                                            const T* __restrict__ b, double sigma, int k,
                                                            const T* __restrict__ V, long long ld,
                                                            T* __restrict__ out, int start, GmresDev sd,
                                                            double* __restrict__ partial) {
  gather_epi_body<T, DIM>(blockIdx.x, gridDim.x, g, ebuf, x, y, b, sigma, k, V, ld, out, start, sd, partial);
}

#include "apply_lines.cuh"

// one launch of the cell kernel: the line form in 3D, the point form in 2D
// (ZP, 3D staged only: the input comes from the star-patch outputs, see PatchIn)
template <typename T, int DIM, bool TENSOR, int MODE, bool STAGED, bool ZP = false>
static void launch_cells(dim3 grid, cudaStream_t s, const Geom& g, const Colour& col, const CellConst<T>& cc,
                         const T* x, T* y, const T* coef, const T* p_in, T* p_out, long long vstride, T* ebuf,
                         const T* winv, PatchIn<T> pin = PatchIn<T>{}) {
  if constexpr (DIM == 3)
    launch_pdl(k_apply_lines<T, TENSOR, MODE, STAGED, ZP>, grid, 256, 0, s, g, col, cc, x, y, coef, p_in, p_out,
               vstride, ebuf, winv, pin);
  else
    launch_pdl(k_apply<T, DIM, TENSOR, MODE, STAGED>, grid, 256, 0, s, g, col, cc, x, y, coef, p_in, p_out, vstride,
               ebuf, winv);
}

template <typename T, int DIM, bool TENSOR, int MODE>
static void launch_apply(const LevelDev& L, double gamma, const void* x, void* y, const void* p_in,
                         void* p_out, int nvec, long long vstride, cudaStream_t s) {
  const Geom& g = L.g;
  constexpr bool NEED_FLUX = (MODE & (OP_VISC | OP_AL | OP_BT)) != 0;
  constexpr int CPB = 8 * (DIM == 2 ? 3 : 1);   // cells per 256-thread block
  const T* coef = nullptr;
  const T* winv = nullptr;
  if constexpr (std::is_same<T, double>::value) { coef = L.coef64; winv = L.winv64; }
  else { coef = L.coef32; winv = L.winv32; }
  const int keep_bnd = ((MODE & OP_VISC) && !(MODE & OP_RAW)) ? 1 : 0;
  if (nvec == 1 && L.ebuf) {
    // one launch over all cells into the per-cell buffer, one gather launch per node
    const Colour col = all_cells(g);
    launch_cells<T, DIM, TENSOR, MODE, true>(dim3((unsigned)((col.count + CPB - 1) / CPB)), s, g, col,
                                             cell_const<T>(g, gamma), (const T*)x, (T*)y, coef, (const T*)p_in,
                                             (T*)p_out, 0, (T*)L.ebuf, winv);
    if (NEED_FLUX) {
      launch_pdl(k_gather_cells<T, DIM>, (gather_threads(g) + 255) / 256, 256, 0, s, g, (const T*)L.ebuf,
                 (const T*)x, (T*)y, keep_bnd, (MODE & OP_RAW) ? 1 : 0);
    }
    count_launch(NEED_FLUX ? 2 : 1);
    return;
  }
  for (int v0 = 0; v0 < nvec; v0 += 65535) {
    const int nv = nvec - v0 < 65535 ? nvec - v0 : 65535;
    const T* xv = (const T*)x + v0 * vstride;
    T* yv = (T*)y + v0 * vstride;
    if (NEED_FLUX) {
      const long long tot = g.N * g.dim;
      dim3 grid((unsigned)((tot + 255) / 256), nv);
      k_init_out<T><<<grid, 256, 0, s>>>(g, xv, yv, keep_bnd, vstride);
    }
    const int ncol = NEED_FLUX ? (1 << DIM) : 1;   // B u alone is cell-local: one launch
    for (int colour = 0; colour < ncol; ++colour) {
      const Colour col = NEED_FLUX ? make_colour(g, colour) : all_cells(g);
      dim3 grid((unsigned)((col.count + CPB - 1) / CPB), nv);
      launch_cells<T, DIM, TENSOR, MODE, false>(grid, s, g, col, cell_const<T>(g, gamma), xv, yv, coef,
                                                (const T*)p_in, (T*)p_out, vstride, nullptr, winv);
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
    case OP_B: launch_apply<T, DIM, TENSOR, OP_B>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
    case OP_BT: launch_apply<T, DIM, TENSOR, OP_BT>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
    default:
      if constexpr (std::is_same<T, double>::value) {
        switch (mode) {
          case OP_VISC | OP_AL | OP_BT | OP_B:
            launch_apply<T, DIM, TENSOR, OP_VISC | OP_AL | OP_BT | OP_B>(L, gamma, x, y, p_in, p_out, nvec, vstride, s);
            break;
          case OP_VISC | OP_AL | OP_RAW:
            launch_apply<T, DIM, TENSOR, OP_VISC | OP_AL | OP_RAW>(L, gamma, x, y, p_in, p_out, nvec, vstride, s);
            break;
          case OP_B | OP_RAW:
            launch_apply<T, DIM, TENSOR, OP_B | OP_RAW>(L, gamma, x, y, p_in, p_out, nvec, vstride, s); break;
          case OP_VISC | OP_BT | OP_B | OP_RAW:   // the nonlinear residual's operators (Newton)
            launch_apply<T, DIM, TENSOR, OP_VISC | OP_BT | OP_B | OP_RAW>(L, gamma, x, y, p_in, p_out, nvec, vstride,
                                                                          s);
            break;
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
  if (L.k == 3) {
    qk_apply(L, prec, mode, gamma, x, y, p_in, p_out, s);
    return;
  }
  op_dispatch(L, prec, mode, gamma, x, y, p_in, p_out, 1, 0, s);
}

template <typename T, int DIM, bool TENSOR>
static void launch_apply_epi(const LevelDev& L, double gamma, const void* x, void* y, const ApplyEpi& e,
                             cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  const Geom& g = L.g;
  constexpr int CPB = 8 * (DIM == 2 ? 3 : 1);
  const T* coef = nullptr;
  const T* winv = nullptr;
  if constexpr (std::is_same<T, double>::value) { coef = L.coef64; winv = L.winv64; }
  else { coef = L.coef32; winv = L.winv32; }
  const Colour col = all_cells(g);
  // External records become event-record nodes when the stream is being captured
  if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
  const dim3 grid((unsigned)((col.count + CPB - 1) / CPB));
  bool fused = false;
  if constexpr (DIM == 3 && std::is_same<T, float>::value) {
    if (e.pout) {   // x = z formed from the patch outputs; z stored on the way
      launch_cells<T, DIM, TENSOR, OP_VISC | OP_AL, true, true>(
          grid, s, g, col, cell_const<T>(g, gamma), nullptr, (T*)y, coef, nullptr, nullptr, 0, (T*)L.ebuf, winv,
          PatchIn<T>{(const T*)e.pout, (const T*)e.pden, (T*)x});
      fused = true;
    }
  }
  if (!fused)
    launch_cells<T, DIM, TENSOR, OP_VISC | OP_AL, true>(grid, s, g, col, cell_const<T>(g, gamma), (const T*)x, (T*)y,
                                                         coef, nullptr, nullptr, 0, (T*)L.ebuf, winv);
  if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
  launch_pdl(k_gather_epi<T, DIM>, (gather_threads(g) + RED_THREADS - 1) / RED_THREADS, RED_THREADS, 0, s, g,
             (const T*)L.ebuf, (const T*)x, (T*)y, (const T*)e.b, e.sigma, e.k, (const T*)e.V, e.ld, (T*)e.out,
             e.start, e.st, e.partial);
  count_launch(2);
}

void op_apply_epi(const LevelDev& L, int prec, double gamma, const void* x, void* y, const ApplyEpi& e,
                  cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  if (L.k == 3) {
    qk_apply_epi(L, prec, gamma, x, y, e, s, e0, e1);
    return;
  }
  if (prec == PREC_F64) {
    if (L.g.dim == 2) {
      if (L.tensor) launch_apply_epi<double, 2, true>(L, gamma, x, y, e, s, e0, e1);
      else launch_apply_epi<double, 2, false>(L, gamma, x, y, e, s, e0, e1);
    } else {
      if (L.tensor) launch_apply_epi<double, 3, true>(L, gamma, x, y, e, s, e0, e1);
      else launch_apply_epi<double, 3, false>(L, gamma, x, y, e, s, e0, e1);
    }
  } else {
    if (L.g.dim == 2) {
      if (L.tensor) launch_apply_epi<float, 2, true>(L, gamma, x, y, e, s, e0, e1);
      else launch_apply_epi<float, 2, false>(L, gamma, x, y, e, s, e0, e1);
    } else {
      if (L.tensor) launch_apply_epi<float, 3, true>(L, gamma, x, y, e, s, e0, e1);
      else launch_apply_epi<float, 3, false>(L, gamma, x, y, e, s, e0, e1);
    }
  }
}

// ---------------------------------------------------------------------------
// merged launches (batch.cuh): FP32, scalar viscosity, 2D and 3D instances in one launch
// (the line form for 3D items, the point form for 2D items, as for a single instance)
// ---------------------------------------------------------------------------
struct CellArgs {
  Geom g;
  Colour col;
  CellConst<float> cc;
  const float* x;
  float* y;
  const float* coef;
  float* ebuf;
  const float* winv;
  PatchIn<float> pin;
};
// ZP: 3D items form x from their star-patch outputs (PatchIn), as op_apply_epi does with
// ApplyEpi::pout; 2D items never do
template <int MODE, bool ZP>
__global__ void __launch_bounds__(256) k_cells_b(const __grid_constant__ BatchTab<CellArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const CellArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i];
  if (a.g.dim == 3)
    apply_lines_body<float, false, MODE, true, ZP>(bx, a.g, a.col, a.cc, a.x, a.y, a.coef, nullptr, nullptr, 0,
                                                   a.ebuf, a.winv, a.pin);
  else
    apply_body<float, 2, false, MODE, true>(bx, a.g, a.col, a.cc, a.x, a.y, a.coef, nullptr, nullptr, 0, a.ebuf,
                                            a.winv);
}

struct GatherArgs {
  Geom g;
  const float* ebuf;
  const float* x;
  float* y;
  const float* b;
  double sigma;
  int k, start, keep_bnd;
  const float* V;
  long long ld;
  float* out;
  GmresDev st;
  double* partial;
};
__global__ void __launch_bounds__(RED_THREADS) k_gather_epi_b(const __grid_constant__ BatchTab<GatherArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const GatherArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i], nb = tb.start[i + 1] - tb.start[i];
  if (a.g.dim == 3)
    gather_epi_body<float, 3>(bx, nb, a.g, a.ebuf, a.x, a.y, a.b, a.sigma, a.k, a.V, a.ld, a.out, a.start, a.st,
                              a.partial);
  else
    gather_epi_body<float, 2>(bx, nb, a.g, a.ebuf, a.x, a.y, a.b, a.sigma, a.k, a.V, a.ld, a.out, a.start, a.st,
                              a.partial);
}
__global__ void __launch_bounds__(256) k_gather_cells_b(const __grid_constant__ BatchTab<GatherArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const GatherArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i];
  if (a.g.dim == 3) gather_cells_body<float, 3>(bx, a.g, a.ebuf, a.x, a.y, a.keep_bnd, 0);
  else gather_cells_body<float, 2>(bx, a.g, a.ebuf, a.x, a.y, a.keep_bnd, 0);
}

static CellArgs cell_args(const BApply& it, bool zp) {
  const LevelDev& L = *it.L;
  CellArgs a{};
  a.g = L.g;
  a.col = all_cells(L.g);
  a.cc = cell_const<float>(L.g, it.gamma);
  a.x = (const float*)it.x;
  a.y = (float*)it.y;
  a.coef = L.coef32;
  a.ebuf = (float*)L.ebuf;
  a.winv = L.winv32;
  if (zp) a.pin = PatchIn<float>{(const float*)it.e.pout, (const float*)it.e.pden, (float*)it.x};
  return a;
}
static unsigned cell_blocks(const Geom& g) {
  const long long cpb = g.dim == 2 ? 24 : 8;
  return (unsigned)((g.ncells + cpb - 1) / cpb);
}

// the cell kernels of every item: 3D items with star-patch input (e.pout) in the ZP
// kernel together with the 2D items, the other 3D items in the plain kernel
template <int MODE>
static int batch_cells(const std::vector<BApply>& items, bool use_pout, cudaStream_t s) {
  std::vector<CellArgs> zp, plain;
  std::vector<unsigned> nzp, nplain;
  bool any_zp = false;
  for (const BApply& it : items) any_zp |= use_pout && it.L->g.dim == 3 && it.e.pout;
  for (const BApply& it : items) {
    const bool z3 = use_pout && it.L->g.dim == 3 && it.e.pout;
    if (z3 || (any_zp && it.L->g.dim == 2)) { zp.push_back(cell_args(it, z3)); nzp.push_back(cell_blocks(it.L->g)); }
    else { plain.push_back(cell_args(it, false)); nplain.push_back(cell_blocks(it.L->g)); }
  }
  int n = 0;
  if (!zp.empty()) n += launch_batch(k_cells_b<MODE, true>, zp, nzp, 256, 0, s);
  if (!plain.empty()) n += launch_batch(k_cells_b<MODE, false>, plain, nplain, 256, 0, s);
  return n;
}

int batch_apply_epi(const std::vector<BApply>& items, cudaStream_t s) {
  int n = batch_cells<OP_VISC | OP_AL>(items, true, s);
  std::vector<GatherArgs> a;
  std::vector<unsigned> nb;
  for (const BApply& it : items) {
    const LevelDev& L = *it.L;
    a.push_back(GatherArgs{L.g, (const float*)L.ebuf, (const float*)it.x, (float*)it.y, (const float*)it.e.b,
                           it.e.sigma, it.e.k, it.e.start, 1, (const float*)it.e.V, it.e.ld, (float*)it.e.out,
                           it.e.st, it.e.partial});
    nb.push_back((gather_threads(L.g) + RED_THREADS - 1) / RED_THREADS);
  }
  n += launch_batch(k_gather_epi_b, a, nb, RED_THREADS, 0, s);
  count_launch(n);
  return n;
}

int batch_apply_al(const std::vector<BApply>& items, cudaStream_t s) {
  int n = batch_cells<OP_AL>(items, false, s);
  std::vector<GatherArgs> a;
  std::vector<unsigned> nb;
  for (const BApply& it : items) {
    const LevelDev& L = *it.L;
    GatherArgs g{};
    g.g = L.g;
    g.ebuf = (const float*)L.ebuf;
    g.x = (const float*)it.x;
    g.y = (float*)it.y;
    g.keep_bnd = 0;   // OP_AL alone: zero Dirichlet rows, as op_apply
    a.push_back(g);
    nb.push_back((gather_threads(L.g) + 255) / 256);
  }
  n += launch_batch(k_gather_cells_b, a, nb, 256, 0, s);
  count_launch(n);
  return n;
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
  if (L.k == 3) {
    qk_load_vector(L, f_qp, F, s);
    return;
  }
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
