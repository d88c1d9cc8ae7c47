// K1, 3D: the cell apply with one lane per (component, 1D line).
//
// Included by operator.cu inside namespace als, after CellConst / Colour / colour_cell.  Same
// arguments and results as k_apply<T, 3, ...>; the difference is the mapping.
// In the point-per-lane form every lane evaluates one Gauss point and reads
// each 1D operand from shared memory, with the 1D tables indexed by the lane's
// runtime coordinates.  Here lane (c, a, b) owns one line of three values of
// velocity component c along the axis being contracted and applies the 3x3
// tables to it in registers, so the table entries are compile-time constants
// (zeros and ones fold away) and three shared-memory values feed six to nine
// FMAs.  Stages (contraction axis, lane = (c, the two other indices)):
//   X:   u -> (B_x u, D_x u)                      (3 global loads per lane)
//   Y:   -> (B_y B_x u, D_y B_x u, B_y D_x u)
//   Z:   -> grad u at the Gauss points, scaled by 2/h
//   point stage: lane = Gauss point: stress, AL projection, fluxes
//   Z^T, Y^T, X^T: the transposed contractions back to the 27 nodes.
// 27 of 32 lanes work; one warp per cell, eight cells per 256-thread block.
#pragma once

template <typename T, int Q, int A>
__device__ __forceinline__ constexpr T cB() { return Ref<T>::B(Q, A); }
template <typename T, int Q, int A>
__device__ __forceinline__ constexpr T cD() { return Ref<T>::D(Q, A); }

// out[q] = sum_a M(q, a) in[a] for the 3x3 table M = B (DER = false) or D (DER = true)
template <typename T, bool DER>
__device__ __forceinline__ void line_fwd(const T (&in)[3], T (&out)[3]) {
  if constexpr (DER) {
    out[0] = cD<T, 0, 0>() * in[0] + cD<T, 0, 1>() * in[1] + cD<T, 0, 2>() * in[2];
    out[1] = cD<T, 1, 0>() * in[0] + cD<T, 1, 1>() * in[1] + cD<T, 1, 2>() * in[2];
    out[2] = cD<T, 2, 0>() * in[0] + cD<T, 2, 1>() * in[1] + cD<T, 2, 2>() * in[2];
  } else {
    out[0] = cB<T, 0, 0>() * in[0] + cB<T, 0, 1>() * in[1] + cB<T, 0, 2>() * in[2];
    out[1] = in[1];                                    // B(1, a) = delta_{a1}
    out[2] = cB<T, 2, 0>() * in[0] + cB<T, 2, 1>() * in[1] + cB<T, 2, 2>() * in[2];
  }
}

// out[a] (+)= sum_q M(q, a) in[q]: the transposed table
template <typename T, bool DER>
__device__ __forceinline__ void line_bwd(const T (&in)[3], T (&out)[3]) {
  if constexpr (DER) {
    out[0] = cD<T, 0, 0>() * in[0] + cD<T, 1, 0>() * in[1] + cD<T, 2, 0>() * in[2];
    out[1] = cD<T, 0, 1>() * in[0] + cD<T, 1, 1>() * in[1] + cD<T, 2, 1>() * in[2];
    out[2] = cD<T, 0, 2>() * in[0] + cD<T, 1, 2>() * in[1] + cD<T, 2, 2>() * in[2];
  } else {
    out[0] = cB<T, 0, 0>() * in[0] + cB<T, 2, 0>() * in[2];
    out[1] = cB<T, 0, 1>() * in[0] + in[1] + cB<T, 2, 1>() * in[2];
    out[2] = cB<T, 0, 2>() * in[0] + cB<T, 2, 2>() * in[2];
  }
}

// Shared-memory layouts of the stage buffers (array m, component c, point or node
// (x, y, z)).  Each buffer is written by one stage and read by the next with the
// lanes spread over different index pairs; these strides were chosen so that the
// 27 lanes of every such access hit 27 distinct banks.
__device__ __forceinline__ int ofs_xy(int m, int c, int x, int y, int z) { return m * 81 + c * 9 + x + 27 * y + 3 * z; }
__device__ __forceinline__ int ofs_yz(int m, int c, int x, int y, int z) { return m * 81 + c * 9 + 3 * x + y + 27 * z; }
__device__ __forceinline__ int ofs_pt(int m, int c, int x, int y, int z) { return m * 81 + c * 27 + 3 * x + 9 * y + z; }

// Input of the apply taken straight from the star-patch outputs (ZP): x = z = (sum of the
// <= 2^d patch outputs containing each node) / den, summed in the fixed order of the patch
// gather (z tap, y tap, then the x pair), 0 at Dirichlet nodes; z is also stored, each node
// by the one cell that owns it (the cell with the node's lower corner, the last cell for the
// upper boundary nodes), so the separate gather launch is not needed.
template <typename T>
struct PatchIn {
  const T* out;   // patch outputs in the row layout (patch_out_index)
  const T* den;   // the GMRES column norm h_j (device scalar)
  T* z;           // z written here
};

// z at the three nodes 2cx + a of the x-line (component c, y node nj, z node nk); 0 on Dirichlet rows
template <typename T>
__device__ __forceinline__ void patch_line(const Geom& g, const PatchIn<T>& pin, T inv_den, int c, int cx, int nj,
                                           int nk, T (&u)[3]) {
  u[0] = u[1] = u[2] = T(0);
  if (nj == 0 || nj == g.nn[1] - 1 || nk == 0 || nk == g.nn[2] - 1) return;
  // taps per axis: odd node 2v+1 -> vertices v (offset 2), v+1 (offset 0); even node 2v -> v (offset 1)
  int vy[2], oy[2], vz[2], oz[2];
  bool oky[2], okz[2];
  if (nj & 1) { vy[0] = nj >> 1; oy[0] = 2; vy[1] = vy[0] + 1; oy[1] = 0; oky[0] = oky[1] = true; }
  else { vy[0] = nj >> 1; oy[0] = 1; oky[0] = true; vy[1] = 0; oy[1] = 0; oky[1] = false; }
  if (nk & 1) { vz[0] = nk >> 1; oz[0] = 2; vz[1] = vz[0] + 1; oz[1] = 0; okz[0] = okz[1] = true; }
  else { vz[0] = nk >> 1; oz[0] = 1; okz[0] = true; vz[1] = 0; oz[1] = 0; okz[1] = false; }
  const int ncol = 3 * g.nv[0];
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int tz = 0; tz < 2; ++tz)
#pragma unroll
    for (int ty = 0; ty < 2; ++ty) {
      if (!(oky[ty] && okz[tz])) continue;
      const int row = ((c * 3 + oz[tz]) * 3 + oy[ty]) * (g.nv[1] * g.nv[2]) + vz[tz] * g.nv[1] + vy[ty];
      const T* rp = pin.out + (long long)row * ncol + 3 * cx;
      const T v1 = rp[1], v2 = rp[2], v3 = rp[3], v4 = rp[4];   // nodes 2cx | 2cx+1 (two) | 2cx+2
      acc[0] += v1;
      acc[1] += v2 + v3;
      acc[2] += v4;
    }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ni = 2 * cx + a;
    u[a] = (ni == 0 || ni == g.nn[0] - 1) ? T(0) : acc[a] * inv_den;
  }
}

template <typename T, bool TENSOR, int MODE, bool STAGED, bool ZP = false>
__device__ __forceinline__ void apply_lines_body(unsigned bx, const Geom& g, const Colour& col, const CellConst<T>& cc,
                                                 const T* __restrict__ x, T* __restrict__ y,
                                                 const T* __restrict__ coef, const T* __restrict__ p_in,
                                                 T* __restrict__ p_out, long long vstride, T* __restrict__ ebuf,
                                                 const T* __restrict__ winv, const PatchIn<T>& pin) {
  constexpr int NB = 27, NPR = 4;
  constexpr int NCQ = TENSOR ? Sz<3>::NC : 1;
  constexpr bool RAW = (MODE & OP_RAW) != 0;
  constexpr bool VISC = (MODE & OP_VISC) != 0;
  constexpr bool NEED_U = (MODE & (OP_VISC | OP_AL | OP_B)) != 0;
  constexpr bool NEED_FLUX = (MODE & (OP_VISC | OP_AL | OP_BT)) != 0;
  // two ping-pong buffers of 3 components x 3 arrays x 27 values per warp
  __shared__ T shA[8][243];
  __shared__ T shB[8][243];
  x += blockIdx.y * vstride;
  y += blockIdx.y * vstride;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* SA = shA[w];
  T* SB = shB[w];
  const bool lane_ok = lane < 27;
  const int c = lane_ok ? lane / 9 : 0;      // velocity component of the line stages
  const int r = lane_ok ? lane % 9 : 0;
  const int b1 = r % 3, b2 = r / 3;          // the two fixed indices of the lane's line
  const long long t = (long long)bx * (blockDim.x >> 5) + w;
  int cx = 0, cy = 0, cz = 0;
  const bool act = colour_cell(col, t, cx, cy, cz);
  // no node of the cell on the boundary: the per-node Dirichlet tests are skipped (warp-uniform)
  const bool inner = cx > 0 && cx < g.n[0] - 1 && cy > 0 && cy < g.n[1] - 1 && cz > 0 && cz < g.n[2] - 1;
  const long long cell = (long long)(unsigned)(cx + g.n[0] * (cy + g.n[1] * cz));
  // point stage: lane = Gauss point (i0, i1, i2)
  const int p = lane_ok ? lane : 0;
  const int i0 = p % 3, i1 = (p / 3) % 3, i2 = p / 9;

  T grad[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) grad[a][k] = T(0);
  pdl_wait();
  // Tensor C (FP32): the cell's 27 x 21 Mandel entries are contiguous; the warp stages them
  // in shared memory with coalesced loads (issued here, beside stage X's loads), and the
  // point stage reads its 21 entries from there (stride 21: every lane a different bank)
  // instead of each lane loading 21 words 84 bytes apart.  (FP64 would exceed the 48 KB
  // of static shared memory per block; it keeps the direct loads.)
  constexpr bool STAGE_C = TENSOR && VISC && sizeof(T) == 4;
  constexpr int CSZ = NB * NCQ;
  __shared__ T shC[STAGE_C ? 8 : 1][STAGE_C ? CSZ : 1];
  if constexpr (STAGE_C) {
    if (act) {
      const T* src = coef + cell * CSZ;
      T v[(CSZ + 31) / 32];
#pragma unroll
      for (int k = 0; k < (CSZ + 31) / 32; ++k) {
        const int e = lane + 32 * k;
        v[k] = e < CSZ ? __ldg(src + e) : T(0);
      }
#pragma unroll
      for (int k = 0; k < (CSZ + 31) / 32; ++k) {
        const int e = lane + 32 * k;
        if (e < CSZ) shC[w][e] = v[k];
      }
    }
  }

  if constexpr (NEED_U) {
    // stage X: lane (c, ay = b1, az = b2) loads the x-line of component c
    {
      T u[3] = {T(0), T(0), T(0)};
      if (act && lane_ok) {
        const int nj = 2 * cy + b1, nk = 2 * cz + b2;
        const long long row = (long long)c * g.N + (long long)(unsigned)(g.nn[0] * (nj + g.nn[1] * nk));
        if constexpr (ZP) {
          const T dn = pin.den[0];
          patch_line<T>(g, pin, dn != T(0) ? T(1) / dn : T(0), c, cx, nj, nk, u);
          // the owned nodes of the line: lower corner, or the last cell for the upper boundary
          if ((b1 < 2 || cy == g.n[1] - 1) && (b2 < 2 || cz == g.n[2] - 1)) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
              if (a < 2 || cx == g.n[0] - 1) pin.z[row + 2 * cx + a] = u[a];
          }
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int ni = 2 * cx + a;
            if (RAW || inner || !on_boundary(g, ni, nj, nk)) u[a] = x[row + ni];
          }
        }
      }
      T bu[3], du[3];
      line_fwd<T, false>(u, bu);
      line_fwd<T, true>(u, du);
      if (lane_ok) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          SA[ofs_xy(0, c, q, b1, b2)] = bu[q];
          SA[ofs_xy(1, c, q, b1, b2)] = du[q];
        }
      }
    }
    __syncwarp();
    // stage Y: lane (c, qx = b1, az = b2)
    if (lane_ok) {
      T v0[3], v1[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        v0[a] = SA[ofs_xy(0, c, b1, a, b2)];
        v1[a] = SA[ofs_xy(1, c, b1, a, b2)];
      }
      T o0[3], o1[3], o2[3];
      line_fwd<T, false>(v0, o0);   // B_y B_x u
      line_fwd<T, true>(v0, o1);    // D_y B_x u
      line_fwd<T, false>(v1, o2);   // B_y D_x u
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        SB[ofs_yz(0, c, b1, q, b2)] = o0[q];
        SB[ofs_yz(1, c, b1, q, b2)] = o1[q];
        SB[ofs_yz(2, c, b1, q, b2)] = o2[q];
      }
    }
    __syncwarp();
    // stage Z: lane (c, qx = b1, qy = b2): gradient of component c at the three points of its z-line
    if (lane_ok) {
      T v0[3], v1[3], v2[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        v0[a] = SB[ofs_yz(0, c, b1, b2, a)];
        v1[a] = SB[ofs_yz(1, c, b1, b2, a)];
        v2[a] = SB[ofs_yz(2, c, b1, b2, a)];
      }
      T gz[3], gy[3], gx[3];
      line_fwd<T, true>(v0, gz);
      line_fwd<T, false>(v1, gy);
      line_fwd<T, false>(v2, gx);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        SA[ofs_pt(0, c, b1, b2, q)] = gx[q] * cc.s[0];
        SA[ofs_pt(1, c, b1, b2, q)] = gy[q] * cc.s[1];
        SA[ofs_pt(2, c, b1, b2, q)] = gz[q] * cc.s[2];
      }
    }
    __syncwarp();
    if (lane_ok) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) grad[a][k] = SA[ofs_pt(k, a, i0, i1, i2)];
    }
  }

  // point stage: weight, pressure basis, divergence moments (warp reduction)
  const T wq = cc.wdet * Ref<T>::W(i0) * Ref<T>::W(i1) * Ref<T>::W(i2);
  T psi[NPR];
  psi[0] = T(1);
  psi[1] = Ref<T>::G(i0);
  psi[2] = Ref<T>::G(i1);
  psi[3] = Ref<T>::G(i2);
  T m[NPR];
#pragma unroll
  for (int q = 0; q < NPR; ++q) m[q] = T(0);
  if constexpr ((MODE & (OP_AL | OP_B)) != 0) {
    T dv = grad[0][0] + grad[1][1] + grad[2][2];
    dv = lane_ok ? wq * dv : T(0);
#pragma unroll
    for (int q = 0; q < NPR; ++q) {
      T v = dv * psi[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      m[q] = v;
    }
    if constexpr ((MODE & OP_B) != 0) {
      if (act && lane < NPR) p_out[cell * NPR + lane] = -m[lane];
    }
  }
  if constexpr (NEED_FLUX) {
    // isotropic part of the stress: gamma Pi div u - p_h
    T pi[NPR];
#pragma unroll
    for (int q = 0; q < NPR; ++q) {
      pi[q] = T(0);
      if constexpr ((MODE & OP_AL) != 0) {
        if (winv) {   // W = M_p(1/mu): per-cell (d+1)^2 block of W^-1
          T acc = T(0);
          if (act) {
#pragma unroll
            for (int k = 0; k < NPR; ++k) acc += winv[(cell * NPR + q) * NPR + k] * m[k];
          }
          pi[q] += cc.gamma * acc;
        } else {      // W = M_p = |K| diag(1, 1/3, ..)
          pi[q] += cc.gamma * m[q] * (q == 0 ? cc.inv_m0 : cc.inv_m1);
        }
      }
      if constexpr ((MODE & OP_BT) != 0) pi[q] -= act ? p_in[cell * NPR + q] : T(0);
    }
    T iso = T(0);
#pragma unroll
    for (int q = 0; q < NPR; ++q) iso += pi[q] * psi[q];
    T sg[3][3];
    if constexpr (VISC) {
      if (act && lane_ok) {
        if constexpr (STAGE_C) stress<T, 3, true>(&shC[w][p * NCQ], grad, iso, sg);
        else stress<T, 3, TENSOR>(coef + (cell * NB + p) * NCQ, grad, iso, sg);
      }
      else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int k = 0; k < 3; ++k) sg[a][k] = T(0);
      }
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) sg[a][k] = (a == k) ? iso : T(0);
    }
    // fluxes F[a][k] = |J| w_q sigma_ak (2/h_k), point-major per (a, k)
    if (lane_ok) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) SB[ofs_pt(k, a, i0, i1, i2)] = wq * sg[a][k] * cc.s[k];
    }
    __syncwarp();
    // stage Z^T: lane (c, qx = b1, qy = b2): P_x = B_z^T F_x, P_y = B_z^T F_y, P_z = D_z^T F_z
    if (lane_ok) {
      T fx[3], fy[3], fz[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        fx[q] = SB[ofs_pt(0, c, b1, b2, q)];
        fy[q] = SB[ofs_pt(1, c, b1, b2, q)];
        fz[q] = SB[ofs_pt(2, c, b1, b2, q)];
      }
      T px[3], py[3], pz[3];
      line_bwd<T, false>(fx, px);
      line_bwd<T, false>(fy, py);
      line_bwd<T, true>(fz, pz);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        SA[ofs_yz(0, c, b1, b2, a)] = px[a];
        SA[ofs_yz(1, c, b1, b2, a)] = py[a];
        SA[ofs_yz(2, c, b1, b2, a)] = pz[a];
      }
    }
    __syncwarp();
    // stage Y^T: lane (c, qx = b1, az = b2): R_x = B_y^T P_x, R_yz = D_y^T P_y + B_y^T P_z
    if (lane_ok) {
      T v0[3], v1[3], v2[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        v0[q] = SA[ofs_yz(0, c, b1, q, b2)];
        v1[q] = SA[ofs_yz(1, c, b1, q, b2)];
        v2[q] = SA[ofs_yz(2, c, b1, q, b2)];
      }
      T rx[3], ry[3], rz[3];
      line_bwd<T, false>(v0, rx);
      line_bwd<T, true>(v1, ry);
      line_bwd<T, false>(v2, rz);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        SB[ofs_xy(0, c, b1, a, b2)] = rx[a];
        SB[ofs_xy(1, c, b1, a, b2)] = ry[a] + rz[a];
      }
    }
    __syncwarp();
    // stage X^T: lane (c, ay = b1, az = b2): y = D_x^T R_x + B_x^T R_yz at the x-line's nodes
    if (lane_ok) {
      T v0[3], v1[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        v0[q] = SB[ofs_xy(0, c, q, b1, b2)];
        v1[q] = SB[ofs_xy(1, c, q, b1, b2)];
      }
      T yd[3], yb[3];
      line_bwd<T, true>(v0, yd);
      line_bwd<T, false>(v1, yb);
      if constexpr (STAGED) {
        // the cell's 27 x-line outputs to shared memory (row = lane); written out below
#pragma unroll
        for (int a = 0; a < 3; ++a) SA[lane * 3 + a] = yd[a] + yb[a];
      } else if (act) {
        {
          const int nj = 2 * cy + b1, nk = 2 * cz + b2;
          const long long row = (long long)c * g.N + (long long)(unsigned)(g.nn[0] * (nj + g.nn[1] * nk));
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int ni = 2 * cx + a;
            if (RAW || inner || !on_boundary(g, ni, nj, nk)) y[row + ni] += yd[a] + yb[a];
          }
        }
      }
    }
    if constexpr (STAGED) {
      // Block write-out in the row layout (stage_row), summed per node by the gather in
      // a fixed order: thread (row rr, cell wc) stores that cell's three values of the
      // row, so the eight cells of a block (consecutive in x when n0 is a multiple of 8)
      // fill one contiguous run of 24 values per row.
      __shared__ int cc_xyz[8][4];
      if (lane == 0) { cc_xyz[w][0] = cx; cc_xyz[w][1] = cy; cc_xyz[w][2] = cz; cc_xyz[w][3] = act ? 1 : 0; }
      __syncthreads();
      if (threadIdx.x < 27 * 8) {
        const int rr = threadIdx.x >> 3, wc = threadIdx.x & 7;
        if (cc_xyz[wc][3]) {
          const int cr = rr / 9, lz = (rr / 3) % 3, ly = rr % 3;
          T* e = ebuf + (long long)stage_row(g, cr, ly, lz, cc_xyz[wc][1], cc_xyz[wc][2]) * (3 * g.n[0]) +
                 3 * cc_xyz[wc][0];
          const T* src = &shA[wc][rr * 3];
          e[0] = src[0];
          e[1] = src[1];
          e[2] = src[2];
        }
      }
    }
  }  // NEED_FLUX
  pdl_trigger();
}
template <typename T, bool TENSOR, int MODE, bool STAGED, bool ZP = false>
__global__ void __launch_bounds__(256) k_apply_lines(Geom g, Colour col, CellConst<T> cc, const T* __restrict__ x,
                                                     T* __restrict__ y, const T* __restrict__ coef,
                                                     const T* __restrict__ p_in, T* __restrict__ p_out,
                                                     long long vstride, T* __restrict__ ebuf,
                                                     const T* __restrict__ winv, PatchIn<T> pin) {
  apply_lines_body<T, TENSOR, MODE, STAGED, ZP>(blockIdx.x, g, col, cc, x, y, coef, p_in, p_out, vstride, ebuf, winv,
                                                pin);
}
