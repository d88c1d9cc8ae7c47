// Shared device-side definitions for the AL-multigrid Stokes library.
//
// Discretisation: [Q2]^d x P1^disc on a uniform mesh of (0,1)^d (Sec. 4 of
// Shih, Stadler & Wechsung, "Robust multigrid techniques for augmented
// Lagrangian preconditioning of incompressible Stokes equations with extreme
// viscosity variations").  Velocity vectors hold d blocks of nodal values on
// the (2n+1)^d Q2 lattice (x fastest); pressures are [cell][d+1] coefficients
// of {1, xi_0, .., xi_(d-1)} on the reference cell [-1,1]^d.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace als {

// ---------------------------------------------------------------- geometry
struct Geom {
  int dim;
  int n[3];      // cells per direction (n[2] = 1 in 2D)
  int nn[3];     // Q2 nodes per direction, 2n+1 (nn[2] = 1 in 2D)
  int nv[3];     // vertices per direction, n+1 (nv[2] = 1 in 2D)
  long long N;   // nodes
  long long ncells;
  long long nverts;
  double h[3];
};

// Reference-element tables on [-1,1], as compile-time formulas: the three
// quadratic Lagrange polynomials l_0 = xi(xi-1)/2, l_1 = 1-xi^2,
// l_2 = xi(xi+1)/2 on the nodes -1, 0, 1 and their derivatives, evaluated at
// the 3-point Gauss-Legendre abscissae (-g, 0, g), g = sqrt(3/5), with weights
// (5/9, 8/9, 5/9).  With g^2 = 3/5: l_0(-g) = l_2(g) = 3/10 + g/2,
// l_2(-g) = l_0(g) = 3/10 - g/2, l_1(+-g) = 2/5.
template <typename T>
struct Ref {
  static constexpr T g = T(0.774596669241483377035853079956);
  __host__ __device__ __forceinline__ static constexpr T G(int q) {
    return q == 0 ? -g : (q == 1 ? T(0) : g);
  }
  __host__ __device__ __forceinline__ static constexpr T W(int q) {
    return q == 1 ? T(8.0 / 9.0) : T(5.0 / 9.0);
  }
  __host__ __device__ __forceinline__ static constexpr T B(int q, int a) {
    return q == 1 ? (a == 1 ? T(1) : T(0))
                  : (a == 1 ? T(0.4) : (((q == 0) == (a == 0)) ? T(0.3) + T(0.5) * g : T(0.3) - T(0.5) * g));
  }
  __host__ __device__ __forceinline__ static constexpr T D(int q, int a) {
    return a == 0 ? G(q) - T(0.5) : (a == 1 ? T(-2) * G(q) : G(q) + T(0.5));
  }
};

// ---------------------------------------------------------------- status
// Device-side failures never trap: kernels record a code and an index here
// and the host reads the record back at the end of setup/solve.
struct DevStatus {
  int code;        // 0 = ok, otherwise an als_status value
  long long where; // e.g. the vertex whose patch matrix had a non-positive pivot
};

__device__ __forceinline__ void report(DevStatus* st, int code, long long where) {
  if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}

__host__ __device__ __forceinline__ bool on_boundary(const Geom& g, int i, int j, int k) {
  if (i == 0 || i == g.nn[0] - 1 || j == 0 || j == g.nn[1] - 1) return true;
  if (g.dim == 3 && (k == 0 || k == g.nn[2] - 1)) return true;
  return false;
}

__host__ __device__ __forceinline__ long long node_id(const Geom& g, int i, int j, int k) {
  return (long long)i + (long long)g.nn[0] * ((long long)j + (long long)g.nn[1] * k);
}

// Row layout of per-cell staged outputs (operator apply, star patches): the
// value a cell (cx, cy, cz) contributes to its local node (lx, ly, lz) of
// component c sits in row ((c L + lz) 3 + ly) n1 n2 + cz n1 + cy at column
// 3 cx + lx, rows of 3 n0 values (L = 3 in 3D, 1 in 2D).  Along a row of
// global nodes x = 0..2 n0 the contributions are then contiguous: node 2i reads
// columns 3i-1 and 3i, node 2i+1 column 3i+1, so a gather over x is a
// streaming read.
__host__ __device__ __forceinline__ int stage_row(const Geom& g, int c, int ly, int lz, int cy, int cz) {
  const int L = g.dim == 3 ? 3 : 1;
  return ((c * L + lz) * 3 + ly) * (g.n[1] * g.n[2]) + cz * g.n[1] + cy;
}

// Row gathers: one thread handles GX consecutive nodes x = GX j .. GX j + GX-1 of
// the node row (component c, y, z).
constexpr int GX = 4;

struct RowChunk {
  int c, y, z, j;
  long long t0;   // vector index of node x = 4j
};

__device__ __forceinline__ bool row_chunk(const Geom& g, int dim, unsigned t, RowChunk& rc) {
  const unsigned cpr = (unsigned)((g.nn[0] + GX - 1) / GX);
  const unsigned rows = (unsigned)(dim * g.nn[1] * g.nn[2]);
  const unsigned row = t / cpr;
  if (row >= rows) return false;
  rc.j = (int)(t - row * cpr);
  const unsigned ny = (unsigned)g.nn[1], nz = (unsigned)g.nn[2];
  const unsigned rz = row / ny;
  rc.y = (int)(row - rz * ny);
  rc.c = (int)(rz / nz);
  rc.z = (int)(rz - (unsigned)rc.c * nz);
  rc.t0 = (long long)rc.c * g.N + ((long long)rc.z * g.nn[1] + rc.y) * g.nn[0] + GX * rc.j;
  return true;
}

// Row layout of vertex-star patch outputs: entry (c, ox, oy, oz) of the patch of
// vertex (vx, vy, vz) (node 2v - 1 + o per axis) sits in row
// ((c L + oz) 3 + oy) nv1 nv2 + vz nv1 + vy at column 3 vx + ox, rows of 3 nv0
// values.  Node 2v reads column 3v+1; node 2v+1 reads columns 3v+2 and 3v+3.
template <int DIM>
__host__ __device__ __forceinline__ long long patch_out_index(const Geom& g, int vx, int vy, int vz, int i) {
  constexpr int NB = DIM == 3 ? 27 : 9;
  const int c = i / NB, o = i - c * NB;
  const int ox = o % 3, oy = (o / 3) % 3, oz = DIM == 3 ? o / 9 : 0;
  const int L = DIM == 3 ? 3 : 1;
  const int row = ((c * L + oz) * 3 + oy) * (g.nv[1] * g.nv[2]) + vz * g.nv[1] + vy;
  return (long long)row * (3 * g.nv[0]) + 3 * vx + ox;
}

template <int DIM> struct Sz;
template <> struct Sz<2> { static constexpr int NB = 9, NP = 18, NPR = 3, NM = 3, NC = 6, NCELL_STAR = 4; };
template <> struct Sz<3> { static constexpr int NB = 27, NP = 81, NPR = 4, NM = 6, NC = 21, NCELL_STAR = 8; };

// packed symmetric storage of an NP x NP patch inverse, by diagonals:
// diagonal t (0..NP-1) holds the entries (i, i+t), i = 0..NP-1-t.
__host__ __device__ constexpr int diag_start(int np, int t) { return t * np - (t * (t - 1)) / 2; }
__host__ __device__ constexpr int packed_size(int np) { return np * (np + 1) / 2; }
// per-patch stride, rounded to a multiple of 4 entries (16-byte aligned rows)
__host__ __device__ constexpr int packed_stride(int np) { return (packed_size(np) + 3) & ~3; }

// "Block-packed" storage of the same symmetric NP x NP matrix (NP = 9 NBR), used
// for the FP32 inverses: 9x9 blocks (I, J), I <= J, numbered off-diagonal blocks
// first (row-major over I < J), then the NBR diagonal blocks.  Element e of a
// block is r*9 + c (off-diagonal, 81 entries) or the row-major index of (r, c),
// r <= c, in the 45-entry upper triangle (diagonal).  Storage is interleaved by
// block in 16-byte quads so that thread b of a patch reads consecutive 16-byte
// words: elements 0..43 of all NBP blocks as 11 quads (quad q of block b at
// 4 (q NBP + b)), then element 44 of all blocks (padded to a multiple of 4
// floats), then elements 45..80 of the off-diagonal blocks as 9 quads.  The
// total is NP (NP + 1) / 2 entries plus that padding (= packed_stride(NP)).
struct BlockLayout {
  int nbr, nbp, noff, q2;
  __host__ __device__ constexpr explicit BlockLayout(int np)
      : nbr(np / 9), nbp((np / 9) * (np / 9 + 1) / 2), noff((np / 9) * (np / 9 - 1) / 2),
        q2(44 * ((np / 9) * (np / 9 + 1) / 2) + ((((np / 9) * (np / 9 + 1) / 2) + 3) & ~3)) {}
  __host__ __device__ constexpr int offdiag(int I, int J) const {  // I < J
    return I * (nbr - 1) - (I * (I - 1)) / 2 + (J - I - 1);
  }
  __host__ __device__ constexpr int slot(int e, int b) const {
    return e < 44 ? 4 * ((e >> 2) * nbp + b) + (e & 3)
                  : (e == 44 ? 44 * nbp + b : q2 + 4 * (((e - 45) >> 2) * noff + b) + ((e - 45) & 3));
  }
  // position of entry (i, j), i <= j
  __host__ __device__ constexpr int index(int i, int j) const {
    const int I = i / 9, r = i % 9, J = j / 9, c = j % 9;
    if (I == J) return slot(r * 9 - (r * (r - 1)) / 2 + (c - r), noff + I);
    return slot(r * 9 + c, offdiag(I, J));
  }
};

}  // namespace als
