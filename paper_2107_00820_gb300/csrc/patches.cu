// K2/K3/K4: vertex-star patches of the PSC smoother (Sec. 4.1, Eq. (viim)).
//
// For every vertex v the local space V_v = {v in V_h : supp v in star(v)} is
// spanned by the free dofs at the 3^d Q2 nodes within half a cell of v.  Its
// matrix A_v is the restriction of the assembled A_(h,gamma) to V_v; here it is
// accumulated directly from the contributions of the 2^d cells of the star and
// inverted by the symmetric sweep operator without pivoting (A_v is SPD; see
// patch_setup.cuh), in FP64 or, for the mixed cycle, in double-float arithmetic;
// the inverse is stored packed (symmetric) in FP64 and block-packed in FP32.
// Missing nodes of boundary stars become identity rows so that every patch has
// d*3^d entries.
//
// The smoother applies z = sum_v I_v A_v^-1 I_v^T r in two deterministic steps:
// the patch kernel computes y_v = A_v^-1 r|_v into a per-patch buffer (row layout),
// then the <= 2^d patch values that contain a node are summed in a fixed order (no
// floating-point atomics) by the patch gather or, in the FP32 3D smoother, by the
// operator's cell kernel that consumes z.
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <type_traits>

#include "df64.cuh"
#include "level.h"
#include "batch.cuh"
#include "pdl.cuh"

namespace als {

// node offset index o in [0, 3^d): offsets (o%3 - 1, (o/3)%3 - 1, o/9 - 1) from 2v
template <int DIM>
__device__ __forceinline__ bool patch_node(const Geom& g, int vx, int vy, int vz, int o, long long& nd) {
  const int i = 2 * vx + o % 3 - 1;
  const int j = 2 * vy + (o / 3) % 3 - 1;
  const int k = (DIM == 3) ? 2 * vz + o / 9 - 1 : 0;
  if (i <= 0 || i >= g.nn[0] - 1 || j <= 0 || j >= g.nn[1] - 1) return false;
  if (DIM == 3 && (k <= 0 || k >= g.nn[2] - 1)) return false;
  nd = node_id(g, i, j, k);
  return true;
}

template <int DIM>
__device__ __forceinline__ void vertex_coords(const Geom& g, long long v, int& vx, int& vy, int& vz) {
  vx = (int)(v % g.nv[0]);
  const long long r = v / g.nv[0];
  vy = (int)(r % g.nv[1]);
  vz = (DIM == 3) ? (int)(r / g.nv[1]) : 0;
}

// Free node offsets of a boundary vertex's star along each axis: all three offsets
// (0, 1, 2) where the vertex is interior along the axis, only the inward one where it
// lies on the boundary (2 at v = 0, 0 at v = n); entries of the star with an offset
// outside [lo, lo + cnt) on some axis are absent or Dirichlet nodes.
template <int DIM>
struct StarAxes {
  int lo[3], cnt[3], m;   // m = free dofs = DIM cnt0 cnt1 cnt2
  __device__ __forceinline__ StarAxes(const Geom& g, int vx, int vy, int vz) {
    const int v[3] = {vx, vy, vz};
    m = DIM;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k >= DIM) { lo[k] = 0; cnt[k] = 1; continue; }
      if (v[k] == 0) { lo[k] = 2; cnt[k] = 1; }
      else if (v[k] == g.nv[k] - 1) { lo[k] = 0; cnt[k] = 1; }
      else { lo[k] = 0; cnt[k] = 3; }
      m *= cnt[k];
    }
  }
  // patch entry (component-major, offsets x-fastest) of free dof a
  __device__ __forceinline__ int entry(int a) const {
    constexpr int NB = Sz<DIM>::NB;
    const int ix = a % cnt[0], q = a / cnt[0], iy = q % cnt[1], q2 = q / cnt[1], iz = q2 % cnt[2], c = q2 / cnt[2];
    return c * NB + (lo[0] + ix) + 3 * (lo[1] + iy) + 9 * (lo[2] + iz);
  }
  // free dof of patch entry i, or -1
  __device__ __forceinline__ int free_index(int i) const {
    constexpr int NB = Sz<DIM>::NB;
    const int c = i / NB, o = i - c * NB;
    const int ix = o % 3 - lo[0], iy = (o / 3) % 3 - lo[1], iz = o / 9 - lo[2];
    if (ix < 0 || ix >= cnt[0] || iy < 0 || iy >= cnt[1] || iz < 0 || iz >= cnt[2]) return -1;
    return ((c * cnt[2] + iz) * cnt[1] + iy) * cnt[0] + ix;
  }
};
__device__ __forceinline__ int tri_pos(int m, int a, int b) { return a * m - (a * (a - 1)) / 2 + (b - a); }  // a <= b

// ---------------------------------------------------------------------------
// K2 + K3: assemble, factor and invert one patch per CTA (FP64)
// ---------------------------------------------------------------------------
// Mandel vector of eps(phi e_al) for grad phi = gr: components (00, 11[, 22], [12, 02,] 01),
// sqrt2 on the shear components
template <int DIM>
__device__ __forceinline__ void mandel_of(int al, const double* gr, double* e) {
  constexpr double ir2 = 0.70710678118654752440;
  if (DIM == 2) {
    e[0] = al == 0 ? gr[0] : 0.0;
    e[1] = al == 1 ? gr[1] : 0.0;
    e[2] = ((al == 0 ? gr[1] : 0.0) + (al == 1 ? gr[0] : 0.0)) * ir2;
  } else {
    e[0] = al == 0 ? gr[0] : 0.0;
    e[1] = al == 1 ? gr[1] : 0.0;
    e[2] = al == 2 ? gr[2] : 0.0;
    e[3] = ((al == 1 ? gr[2] : 0.0) + (al == 2 ? gr[1] : 0.0)) * ir2;
    e[4] = ((al == 0 ? gr[2] : 0.0) + (al == 2 ? gr[0] : 0.0)) * ir2;
    e[5] = ((al == 0 ? gr[1] : 0.0) + (al == 1 ? gr[0] : 0.0)) * ir2;
  }
}

#include "patch_setup.cuh"

// ---------------------------------------------------------------------------
// K4 (FP32): TMA-pipelined block-packed patch products
//
// Persistent CTAs of 128 threads.  Each iteration handles PPI patches whose
// block-packed inverses (see BlockLayout) are streamed into a ring of NSTAGE
// shared-memory stages by 1D bulk copies (cp.async.bulk, completion counted on
// an mbarrier), issued by thread 0 NSTAGE iterations ahead.  Thread b of a
// patch owns one 9x9 block S_IJ and forms both S_IJ r_J and S_IJ^T r_I from
// registers, so each stored entry is read from shared memory exactly once; a
// fixed-order reduction of the block partials gives y_v = A_v^-1 r|_v.
// Every mbarrier wait is bounded: on expiry the kernel records ALS_ETIMEOUT,
// waits (bounded) for the copies it issued and returns.
// ---------------------------------------------------------------------------
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: at most `polls` polls with back-off (the default, kWaitPolls = 2^22, is
// well over a second), false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int polls = kWaitPolls) {
  for (int it = 0; it < polls; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 64) __nanosleep(256);
  }
  return false;
}
__device__ __forceinline__ void fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

}  // namespace tma

enum PatchOut { OUT_SCRATCH = 0, OUT_WRITE = 1, OUT_SUBTRACT = 2 };

// S_IJ r_J -> yI and S_IJ^T r_I -> yJ for block b of one block-packed patch at S
// (global or shared memory).  Diagonal blocks use the symmetric upper triangle.
// Storage of the block-packed FP32-cycle inverses: float, or bfloat16 (the opt-in
// ALS_STORE_BF16) widened to float on load; every product and sum runs in float.
template <bool GLOBAL>
__device__ __forceinline__ float4 ld4(const float* p) {
  if constexpr (GLOBAL) return __ldg(reinterpret_cast<const float4*>(p));
  else return *reinterpret_cast<const float4*>(p);
}
template <bool GLOBAL>
__device__ __forceinline__ float ld1(const float* p) {
  if constexpr (GLOBAL) return __ldg(p);
  else return *p;
}
template <bool GLOBAL>
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {   // four entries, one 8-byte load
  uint2 u;
  if constexpr (GLOBAL) u = __ldg(reinterpret_cast<const uint2*>(p));
  else u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 c = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, c.x, c.y);
}
template <bool GLOBAL>
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) {
  if constexpr (GLOBAL) return __bfloat162float(__ldg(p));
  else return __bfloat162float(*p);
}

// entries per patch of the block-packed layout in storage TS: the packed size rounded to
// 16 bytes (bulk copies and vector loads need 16-byte aligned rows)
template <typename TS>
__host__ __device__ constexpr int block_stride(int np) {
  return sizeof(TS) == 4 ? packed_stride(np) : (packed_size(np) + 7) & ~7;
}

template <bool GLOBAL, typename TS = float>
__device__ __forceinline__ void block_product(const BlockLayout& BL, const TS* __restrict__ S, int b, bool diag,
                                              const float (&rI)[9], const float (&rJ)[9], float (&yI)[9],
                                              float (&yJ)[9]) {
  float e[84];
#pragma unroll
  for (int q = 0; q < 11; ++q) {
    const float4 v = ld4<GLOBAL>(S + 4 * (q * BL.nbp + b));
    e[4 * q] = v.x; e[4 * q + 1] = v.y; e[4 * q + 2] = v.z; e[4 * q + 3] = v.w;
  }
  e[44] = ld1<GLOBAL>(S + 44 * BL.nbp + b);
  if (!diag) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const float4 v = ld4<GLOBAL>(S + BL.q2 + 4 * (q * BL.noff + b));
      e[45 + 4 * q] = v.x; e[46 + 4 * q] = v.y; e[47 + 4 * q] = v.z; e[48 + 4 * q] = v.w;
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) { yI[k] = 0.f; yJ[k] = 0.f; }
  if (diag) {
#pragma unroll
    for (int rr = 0; rr < 9; ++rr)
#pragma unroll
      for (int cc = rr; cc < 9; ++cc) {
        const float sv = e[rr * 9 - (rr * (rr - 1)) / 2 + (cc - rr)];
        yI[rr] += sv * rI[cc];
        if (cc != rr) yI[cc] += sv * rI[rr];
      }
  } else {
    float yI2[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) yI2[k] = 0.f;
#pragma unroll
    for (int rr = 0; rr < 9; ++rr)
#pragma unroll
      for (int cc = 0; cc < 9; ++cc) {
        const float sv = e[rr * 9 + cc];
        if (cc & 1) yI2[rr] += sv * rJ[cc];   // two independent partial sums per row
        else yI[rr] += sv * rJ[cc];
        yJ[cc] += sv * rI[rr];
      }
#pragma unroll
    for (int k = 0; k < 9; ++k) yI[k] += yI2[k];
  }
}

__device__ __forceinline__ void block_of(const BlockLayout& BL, int b, int& I, int& J, bool& diag) {
  diag = b >= BL.noff;
  I = 0;
  J = 0;
  if (diag) {
    I = J = b - BL.noff;
  } else {
    int rem = b;
    while (rem >= BL.nbr - 1 - I) { rem -= BL.nbr - 1 - I; ++I; }
    J = I + 1 + rem;
  }
}

template <int DIM, int NST, typename TS = float>
struct TmaCfg {
  static constexpr int NP = Sz<DIM>::NP;
  static constexpr int NB = Sz<DIM>::NB;
  static constexpr int THREADS = 64;
  static constexpr int TPP = DIM == 3 ? 64 : 4;        // threads per patch (>= blocks per patch)
  static constexpr int PPI = THREADS / TPP;            // patches per iteration
  static constexpr int NSTAGE = NST;
  static constexpr int STRIDE = block_stride<TS>(NP);  // entries per patch
  static constexpr int NBR = NP / 9;
  static constexpr int RPT = (PPI * NP + THREADS - 1) / THREADS;   // r values gathered per thread
  static constexpr size_t stage_elems = (size_t)PPI * STRIDE;
  static constexpr size_t stage_bytes = stage_elems * sizeof(TS);
  // dynamic shared memory: [mbarriers | stages | r | partials]; the barriers need
  // 8-byte and the bulk-copy destinations 16-byte alignment
  static constexpr size_t bar_bytes = 128;
  static constexpr size_t smem_bytes =
      bar_bytes + NSTAGE * stage_bytes + (size_t)PPI * NP * 4 + (size_t)PPI * NP * NBR * 4;
  static_assert(NSTAGE * 8 <= bar_bytes, "mbarrier area too small");
  static_assert((STRIDE * sizeof(TS)) % 16 == 0 && stage_bytes % 16 == 0, "bulk copies need 16-byte alignment");
};

// Work list of the FP32 star kernels, wl = bit 0 | bit 1: bit 0 clear = the star products
// of the smoother, set = the local solves on the coarse-cell interiors (the stars of the
// fine vertices 2K+1 at the coarse-cell centres, which are interior vertices); bit 1 set =
// split storage, where inv32 holds the interior vertices only (interior index x-fastest)
// and the smoother's list is the interior vertices, else inv32 holds every vertex (identity
// rows at absent nodes) and the smoother's list is every vertex.  Returns the index of slot
// p's inverse in inv32 and its lattice coordinates; -1 past the end.
template <int DIM>
__device__ __forceinline__ int work_vertex(const Geom& g, int wl, int p, int count, int& vx, int& vy, int& vz) {
  if (p >= count) return -1;
  const bool split = (wl & 2) != 0;
  const int nix = g.nv[0] - 2, niy = g.nv[1] - 2;
  if (!(wl & 1)) {
    const int ox = split ? 1 : 0, nx = split ? nix : g.nv[0], ny = split ? niy : g.nv[1];
    vx = p % nx + ox;
    const int q = p / nx;
    vy = q % ny + ox;
    vz = DIM == 3 ? q / ny + ox : 0;
    return p;
  }
  const int ncx = g.n[0] >> 1, ncy = g.n[1] >> 1;
  const int kx = p % ncx, q = p / ncx, ky = q % ncy, kz = DIM == 3 ? q / ncy : 0;
  vx = 2 * kx + 1;
  vy = 2 * ky + 1;
  vz = DIM == 3 ? 2 * kz + 1 : 0;
  if (split) return (vx - 1) + nix * ((vy - 1) + (DIM == 3 ? niy * (vz - 1) : 0));
  return vx + g.nv[0] * (vy + g.nv[1] * vz);
}

// r at patch entry i of the vertex (absent nodes give 0)
template <int DIM>
__device__ __forceinline__ float patch_r(const Geom& g, const float* __restrict__ r, int vid, int vx, int vy, int vz,
                                         int i) {
  constexpr int NB = Sz<DIM>::NB;
  if (vid < 0) return 0.f;
  long long nd;
  return patch_node<DIM>(g, vx, vy, vz, i % NB, nd) ? __ldg(r + (i / NB) * g.N + nd) : 0.f;
}

// One patch per iteration (3D): the index arithmetic of a thread's entries is split
// into a per-entry part, fixed for the whole launch, and a per-patch part, formed
// once per patch.  Entry i = c NB + o of the patch of vertex v sits at vector index
// c N + node(2v - 1 + o) and at scratch index patch_out_index(v, i).
struct EntryConst {
  int ox, oy, oz;     // node offsets 0..2 per axis
  int goff;           // c N + (oz - 1) nn0 nn1 + (oy - 1) nn0 + (ox - 1)
  int ooff;           // ((c L + oz) 3 + oy) nv1 nv2 (3 nv0) + ox
  bool ok;            // the thread owns this entry
};
struct PatchPos {
  int vid, vx, vy, vz;
  bool inner;         // no node of the patch on or beyond the boundary
  int gbase;          // node index of 2v
  int obase;          // (vz nv1 + vy) (3 nv0) + 3 vx
};
// (32-bit offsets: vector and scratch lengths stay below 2^31, checked when a context is created)
template <int DIM>
__device__ __forceinline__ EntryConst entry_const(const Geom& g, int e, int total) {
  constexpr int NB = Sz<DIM>::NB;
  EntryConst c{};
  c.ok = e < total;
  const int i = c.ok ? e % Sz<DIM>::NP : 0;
  const int comp = i / NB, o = i - comp * NB;
  c.ox = o % 3;
  c.oy = (o / 3) % 3;
  c.oz = DIM == 3 ? o / 9 : 1;
  const int nn01 = g.nn[0] * g.nn[1];
  c.goff = comp * (int)g.N + (c.oz - 1) * nn01 + (c.oy - 1) * g.nn[0] + (c.ox - 1);
  const int L = DIM == 3 ? 3 : 1;
  const int oz = DIM == 3 ? c.oz : 0;
  c.ooff = ((comp * L + oz) * 3 + c.oy) * (g.nv[1] * g.nv[2]) * (3 * g.nv[0]) + c.ox;
  return c;
}
template <int DIM>
__device__ __forceinline__ PatchPos patch_pos(const Geom& g, int interior, int p, int count) {
  PatchPos q{};
  q.vid = work_vertex<DIM>(g, interior, p, count, q.vx, q.vy, q.vz);
  q.inner = q.vx >= 1 && q.vx <= g.nv[0] - 2 && q.vy >= 1 && q.vy <= g.nv[1] - 2 &&
            (DIM == 2 || (q.vz >= 1 && q.vz <= g.nv[2] - 2));
  q.gbase = 2 * q.vx + 2 * q.vy * g.nn[0] + (DIM == 3 ? 2 * q.vz * g.nn[0] * g.nn[1] : 0);
  q.obase = (q.vz * g.nv[1] + q.vy) * (3 * g.nv[0]) + 3 * q.vx;
  return q;
}
// the node of entry c of the patch at q exists (inside the free nodes)
template <int DIM>
__device__ __forceinline__ bool entry_in(const Geom& g, const PatchPos& q, const EntryConst& c) {
  if (q.inner) return true;
  const int i = 2 * q.vx + c.ox - 1, j = 2 * q.vy + c.oy - 1;
  if (i <= 0 || i >= g.nn[0] - 1 || j <= 0 || j >= g.nn[1] - 1) return false;
  if (DIM == 3) {
    const int k = 2 * q.vz + c.oz - 1;
    if (k <= 0 || k >= g.nn[2] - 1) return false;
  }
  return true;
}

// (bx, gx: the block's index and the blocks of this instance, see batch.cuh)
template <int DIM, int NST, typename TS = float>
__device__ __forceinline__ void patch_tma_body(unsigned bx, unsigned gx, const Geom& g, const TS* __restrict__ inv,
                                               int interior, int count, const float* __restrict__ r,
                                               float* __restrict__ out, int mode, DevStatus* st, int wait_polls,
                                               int early_trigger) {
  using C = TmaCfg<DIM, NST, TS>;
  constexpr int NP = C::NP, NB = C::NB, PPI = C::PPI, TPP = C::TPP, NSTAGE = C::NSTAGE, NBR = C::NBR;
  constexpr int RPT = C::RPT, THREADS = C::THREADS;
  constexpr BlockLayout BL = BlockLayout(NP);
  constexpr int ISSUER = THREADS - 1;                     // idle in the block phase (b >= NBP)
  static_assert(ISSUER % TPP >= BlockLayout(NP).nbp, "the issuing thread must not own a block");
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
  TS* stages = reinterpret_cast<TS*>(smraw + C::bar_bytes);
  float* rs = reinterpret_cast<float*>(smraw + C::bar_bytes + NSTAGE * C::stage_bytes);   // [PPI][NP]
  float* part = rs + PPI * NP;                            // [PPI][NP][NBR]
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int ngroups = (count + PPI - 1) / PPI;

  auto issue = [&](int grp, int stage) {   // one bulk copy per patch of the group
    uint32_t bytes = 0;
    int vids[PPI];
    for (int ps = 0; ps < PPI; ++ps) {
      int vx, vy, vz;
      vids[ps] = work_vertex<DIM>(g, interior, grp * PPI + ps, count, vx, vy, vz);
      if (vids[ps] >= 0) bytes += C::STRIDE * sizeof(TS);
    }
    tma::mbar_expect_tx(&bars[stage], bytes);
    for (int ps = 0; ps < PPI; ++ps)
      if (vids[ps] >= 0)
        tma::bulk_load(stages + stage * C::stage_elems + (size_t)ps * C::STRIDE,
                       inv + (long long)vids[ps] * C::STRIDE, C::STRIDE * sizeof(TS), &bars[stage]);
  };
  auto gather = [&](int grp, float (&v)[RPT]) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int e = tid + k * THREADS;
      v[k] = 0.f;
      if (e < PPI * NP && grp < ngroups) {
        int vx, vy, vz;
        const int vid = work_vertex<DIM>(g, interior, grp * PPI + e / NP, count, vx, vy, vz);
        v[k] = patch_r<DIM>(g, r, vid, vx, vy, vz, e % NP);
      }
    }
  };
  // PPI == 1: the thread's entries all belong to the iteration's one patch
  EntryConst ec[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) ec[k] = entry_const<DIM>(g, tid + k * THREADS, PPI * NP);
  auto gather1 = [&](const PatchPos& q, float (&v)[RPT]) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      v[k] = 0.f;
      if (ec[k].ok && q.vid >= 0 && entry_in<DIM>(g, q, ec[k])) v[k] = __ldg(r + (q.gbase + ec[k].goff));
    }
  };

  if (tid == ISSUER) {
    s_fail = 0;
    for (int i = 0; i < NSTAGE; ++i) tma::mbar_init(&bars[i], 1);
    tma::fence_init();
  }
  __syncthreads();
  if (tid == ISSUER)
    for (int i = 0; i < NSTAGE; ++i) {
      const int grp = bx + i * gx;
      if (grp < ngroups) issue(grp, i);
    }
  // the first inverse blocks (written only by the setup) are in flight; r comes from
  // the preceding kernel of the cycle
  pdl_wait();
  // early_trigger: the successor (the boundary-star kernel, which needs nothing this
  // kernel writes) may start now and run beside this one
  if (early_trigger) pdl_trigger();
  float rpre[RPT];
  PatchPos qcur{}, qnext{};
  if constexpr (PPI == 1) {
    qnext = patch_pos<DIM>(g, interior, bx, count);
    gather1(qnext, rpre);
  } else {
    gather(bx, rpre);
  }

  const int ps = tid / TPP, b = tid % TPP;
  int I = 0, J = 0;
  bool diag = false;
  if (b < BL.nbp) block_of(BL, b, I, J, diag);
  int it = 0;
  for (int grp = bx; grp < ngroups; grp += gx, ++it) {
    const int stage = it % NSTAGE;
    const uint32_t parity = (uint32_t)((it / NSTAGE) & 1);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int e = tid + k * THREADS;
      if (e < PPI * NP) rs[e] = rpre[k];
    }
    // next group's r: in flight while this one is computed
    if constexpr (PPI == 1) {
      qcur = qnext;
      qnext = patch_pos<DIM>(g, interior, grp + gx, count);
      gather1(qnext, rpre);
    } else {
      gather(grp + gx, rpre);
    }
    if (!tma::mbar_wait(&bars[stage], parity, wait_polls)) {
      if (tid == ISSUER) { report(st, 7 /* ALS_ETIMEOUT */, grp); s_fail = 1; }
    }
    __syncthreads();                        // (A) r and the stage are visible
    if (s_fail) break;
    if (b < BL.nbp) {
      const TS* S = stages + stage * C::stage_elems + (size_t)ps * C::STRIDE;
      float rI[9], rJ[9], yI[9], yJ[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        rI[k] = rs[ps * NP + 9 * I + k];
        rJ[k] = rs[ps * NP + 9 * J + k];
      }
      block_product<false, TS>(BL, S, b, diag, rI, rJ, yI, yJ);
      float* pp = part + ps * NP * NBR;
#pragma unroll
      for (int k = 0; k < 9; ++k) pp[(9 * I + k) * NBR + J] = yI[k];
      if (!diag) {
#pragma unroll
        for (int k = 0; k < 9; ++k) pp[(9 * J + k) * NBR + I] = yJ[k];
      }
    }
    __syncthreads();                        // (B) the stage is consumed, the partials are complete
    if (tid == ISSUER) {                    // refill the stage NSTAGE groups ahead
      const int nxt = grp + NSTAGE * gx;
      if (nxt < ngroups) {
        tma::fence_async();
        issue(nxt, stage);
      }
    }
    // y_i = sum_J partial(i, J), fixed order
    if constexpr (PPI == 1) {
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        if (!ec[k].ok || qcur.vid < 0) continue;
        const int i = tid + k * THREADS;
        float acc = 0.f;
#pragma unroll
        for (int jb = 0; jb < NBR; ++jb) acc += part[i * NBR + jb];
        if (mode == OUT_SCRATCH) {
          out[qcur.obase + ec[k].ooff] = acc;
        } else if (entry_in<DIM>(g, qcur, ec[k])) {
          float* o = out + (qcur.gbase + ec[k].goff);
          *o = mode == OUT_SUBTRACT ? *o - acc : acc;
        }
      }
    } else {
      for (int e = tid; e < PPI * NP; e += THREADS) {
        const int p = e / NP, i = e % NP;
        int vx, vy, vz;
        const int v = work_vertex<DIM>(g, interior, grp * PPI + p, count, vx, vy, vz);
        if (v < 0) continue;
        float acc = 0.f;
#pragma unroll
        for (int jb = 0; jb < NBR; ++jb) acc += part[(p * NP + i) * NBR + jb];
        if (mode == OUT_SCRATCH) {
          out[patch_out_index<DIM>(g, vx, vy, vz, i)] = acc;
        } else {
          long long nd;
          if (patch_node<DIM>(g, vx, vy, vz, i % NB, nd)) {
            float* o = out + (i / NB) * g.N + nd;
            *o = mode == OUT_SUBTRACT ? *o - acc : acc;
          }
        }
      }
    }
    // no third barrier: r is read only between (A) and (B) of an iteration and
    // rewritten after (B); the partials are read after (B) and rewritten only after
    // barrier (A) of the next iteration, which every thread reaches after its reads
  }
  if (!early_trigger) pdl_trigger();
  if (s_fail && tid == ISSUER) {
    // drain: wait (bounded, at the default limit whatever wait_polls is) for every copy
    // this CTA issued and did not consume, so that none is in flight when the CTA exits
    int k = it;
    for (int grp = bx + it * gx; grp < ngroups && k < it + NSTAGE; grp += gx, ++k)
      tma::mbar_wait(&bars[k % NSTAGE], (uint32_t)((k / NSTAGE) & 1));
  }
}

template <int DIM, int NST, typename TS = float>
__global__ void __launch_bounds__(64) k_patch_tma(Geom g, const TS* __restrict__ inv, int interior, int count,
                                                  const float* __restrict__ r, float* __restrict__ out, int mode,
                                                  DevStatus* st, int wait_polls, int early_trigger) {
  patch_tma_body<DIM, NST, TS>(blockIdx.x, gridDim.x, g, inv, interior, count, r, out, mode, st, wait_polls,
                               early_trigger);
}

// ---------------------------------------------------------------------------
// K4 (FP32), direct variant: each thread streams its 9x9 block of the
// block-packed inverse straight from global memory with coalesced 16-byte
// loads (thread b of a patch reads consecutive words), gathers its r_I, r_J
// itself, and the block partials are reduced through double-buffered shared
// memory: one barrier per iteration, 2 (3D) or 32 (2D) patches per 128-thread CTA.
// ---------------------------------------------------------------------------
template <int DIM, typename TS = float>
struct DirCfg {
  static constexpr int NP = Sz<DIM>::NP;
  static constexpr int THREADS = 128;
  static constexpr int TPP = DIM == 3 ? 64 : 4;
  static constexpr int PPC = THREADS / TPP;
  static constexpr int NBR = NP / 9;
  static constexpr int STRIDE = block_stride<TS>(NP);
};

// r at entry 9*IB + k (k < 9) of the patch of vertex (vx, vy, vz)
template <int DIM>
__device__ __forceinline__ void gather9(const Geom& g, const float* __restrict__ r, int vx, int vy, int vz, int IB,
                                        float (&out)[9]) {
  constexpr int NB = Sz<DIM>::NB;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int i = 9 * IB + k;
    long long nd;
    out[k] = patch_node<DIM>(g, vx, vy, vz, i % NB, nd) ? __ldg(r + (i / NB) * g.N + nd) : 0.f;
  }
}

template <int DIM, typename TS = float>
__device__ __forceinline__ void patch_direct_body(unsigned bx, unsigned gx, const Geom& g, const TS* __restrict__ inv,
                                                  int interior, int count, const float* __restrict__ r,
                                                  float* __restrict__ out, int mode) {
  using C = DirCfg<DIM, TS>;
  constexpr int NP = C::NP, NB = Sz<DIM>::NB, PPC = C::PPC, TPP = C::TPP, NBR = C::NBR;
  constexpr BlockLayout BL = BlockLayout(NP);
  __shared__ float part[2][PPC][NP][NBR];
  const int tid = threadIdx.x, ps = tid / TPP, b = tid % TPP;
  const int ngroups = (count + PPC - 1) / PPC;
  int buf = 0;
  int I = 0, J = 0;
  bool diag = false;
  if (b < BL.nbp) block_of(BL, b, I, J, diag);
  pdl_wait();
  for (int grp = bx; grp < ngroups; grp += gx, buf ^= 1) {
    if (b < BL.nbp) {
      int vx, vy, vz;
      const int v = work_vertex<DIM>(g, interior, grp * PPC + ps, count, vx, vy, vz);
      if (v >= 0) {
        float rI[9], rJ[9], yI[9], yJ[9];
        gather9<DIM>(g, r, vx, vy, vz, I, rI);
        gather9<DIM>(g, r, vx, vy, vz, J, rJ);
        block_product<true, TS>(BL, inv + (long long)v * C::STRIDE, b, diag, rI, rJ, yI, yJ);
#pragma unroll
        for (int k = 0; k < 9; ++k) part[buf][ps][9 * I + k][J] = yI[k];
        if (!diag) {
#pragma unroll
          for (int k = 0; k < 9; ++k) part[buf][ps][9 * J + k][I] = yJ[k];
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < PPC * NP; e += C::THREADS) {
      const int p = e / NP, i = e % NP;
      int vx, vy, vz;
      const int v = work_vertex<DIM>(g, interior, grp * PPC + p, count, vx, vy, vz);
      if (v < 0) continue;
      float acc = 0.f;
#pragma unroll
      for (int jb = 0; jb < NBR; ++jb) acc += part[buf][p][i][jb];
      if (mode == OUT_SCRATCH) {
        out[patch_out_index<DIM>(g, vx, vy, vz, i)] = acc;
      } else {
        long long nd;
        if (patch_node<DIM>(g, vx, vy, vz, i % NB, nd)) {
          float* o = out + (i / NB) * g.N + nd;
          *o = mode == OUT_SUBTRACT ? *o - acc : acc;
        }
      }
    }
  }
}

template <int DIM, typename TS = float>
__global__ void __launch_bounds__(128) k_patch_direct(Geom g, const TS* __restrict__ inv, int interior, int count,
                                                      const float* __restrict__ r, float* __restrict__ out,
                                                      int mode) {
  patch_direct_body<DIM, TS>(blockIdx.x, gridDim.x, g, inv, interior, count, r, out, mode);
}

template <int DIM>
static void launch_patch_direct(const LevelDev& L, int interior, long long count, const float* r, float* out, int mode,
                                cudaStream_t s) {
  using C = DirCfg<DIM>;
  const long long groups = (count + C::PPC - 1) / C::PPC;
  const long long cap = 152LL * 8;
  const long long grid = groups < cap ? groups : cap;
  if (grid <= 0) return;
  if (L.inv16)
    launch_pdl(k_patch_direct<DIM, __nv_bfloat16>, (unsigned)grid, C::THREADS, 0, s, L.g,
               (const __nv_bfloat16*)L.inv16, interior | (L.split ? 2 : 0), (int)count, r, out, mode);
  else
    launch_pdl(k_patch_direct<DIM>, (unsigned)grid, C::THREADS, 0, s, L.g, L.inv32, interior | (L.split ? 2 : 0),
               (int)count, r, out, mode);
  count_launch(1);
}

// ---------------------------------------------------------------------------
// K4 (FP32), boundary stars: y_v = A_v^-1 r|_v restricted to the free dofs of the
// star (a face, edge or corner vertex has 1/3, 1/9 or 1/27 of the interior star's free
// dofs in 3D), from the compact packed inverses, one warp per boundary vertex; every
// entry of the vertex's scratch row is written (0 at absent and Dirichlet nodes).
//
// It is launched right after the interior-star kernel of the same products and runs
// beside it: that kernel lets it start once its own dependency wait has returned (r is
// then complete, and this kernel reads it from L2), the two write disjoint scratch
// rows, and this kernel waits for its predecessor only at its end, so that its
// successor, which waits for it, sees both kernels' rows.
// ---------------------------------------------------------------------------
// One warp per boundary star (8 per CTA): the star's packed block and r are staged in
// shared memory by all lanes (independent loads), then the rows are formed from there.
template <int DIM>
__device__ __forceinline__ void patch_bnd_body(unsigned bx, unsigned gx, const Geom& g, const float* __restrict__ bnd32,
                                               const int* __restrict__ bvid, const long long* __restrict__ boff,
                                               long long nb, const float* __restrict__ r, float* __restrict__ out) {
  constexpr int NP = Sz<DIM>::NP, NB = Sz<DIM>::NB, MMAX = DIM == 3 ? 27 : 6, SMAX = MMAX * (MMAX + 1) / 2;
  __shared__ float Ss[8][SMAX];
  __shared__ float rs[8][MMAX];
  __shared__ float ys[8][MMAX];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long b = (long long)bx * 8 + w; b < nb; b += (long long)gx * 8) {
    const int v = __ldg(bvid + b);
    const float* S = bnd32 + __ldg(boff + b);
    int vx, vy, vz;
    vertex_coords<DIM>(g, v, vx, vy, vz);
    const StarAxes<DIM> ax(g, vx, vy, vz);
    const int m = ax.m, sz = m * (m + 1) / 2;
    for (int e = lane; e < sz; e += 32) Ss[w][e] = __ldg(S + e);
    if (lane < m) {
      long long nd;
      const int i = ax.entry(lane);
      rs[w][lane] = patch_node<DIM>(g, vx, vy, vz, i % NB, nd) ? __ldcg(r + (i / NB) * g.N + nd) : 0.f;
    }
    __syncwarp();
    if (lane < m) {
      float acc = 0.f;
#pragma unroll 4
      for (int c = 0; c < m; ++c) {
        const int lo = lane < c ? lane : c, hi = lane < c ? c : lane;
        acc += Ss[w][tri_pos(m, lo, hi)] * rs[w][c];
      }
      ys[w][lane] = acc;
    }
    __syncwarp();
    for (int i = lane; i < NP; i += 32) {
      const int a = ax.free_index(i);
      out[patch_out_index<DIM>(g, vx, vy, vz, i)] = a >= 0 ? ys[w][a] : 0.f;
    }
    __syncwarp();
  }
  pdl_wait();
  pdl_trigger();
}

template <int DIM>
__global__ void __launch_bounds__(256) k_patch_bnd(Geom g, const float* __restrict__ bnd32,
                                                   const int* __restrict__ bvid, const long long* __restrict__ boff,
                                                   long long nb, const float* __restrict__ r, float* __restrict__ out) {
  patch_bnd_body<DIM>(blockIdx.x, gridDim.x, g, bnd32, bvid, boff, nb, r, out);
}

template <int DIM>
static void launch_patch_bnd(const LevelDev& L, const float* r, float* out, cudaStream_t s) {
  if (L.nbnd <= 0) return;
  const long long want = (L.nbnd + 7) / 8, cap = 152LL * 16;
  launch_pdl(k_patch_bnd<DIM>, (unsigned)(want < cap ? want : cap), 256, 0, s, L.g, (const float*)L.bnd32,
             (const int*)L.bvid, (const long long*)L.boff, L.nbnd, r, out);
  count_launch(1);
}

// FP32 patch-product kernel variants: 0 = TMA ring with 2 stages, 1 = TMA ring
// with 3 stages, 2 = direct 16-byte loads.  A level uses L.patch_kernel (picked by
// patch_autotune); the environment variable ALS_PATCH_KERNEL = tma2 | tma3 | direct
// forces one for every level.
static int forced_patch_kernel() {
  static int v = -2;
  if (v == -2) {
    const char* e = getenv("ALS_PATCH_KERNEL");
    v = -1;
    if (e && e[0] == 'd') v = 2;
    else if (e && e[0] == 't' && e[3] == '3') v = 1;
    else if (e && e[0] == 't') v = 0;
  }
  return v;
}

static int patch_variant(const LevelDev& L) {
  const int f = forced_patch_kernel();
  if (f >= 0) return f;
  return L.patch_kernel >= 0 ? L.patch_kernel : 0;
}

template <int DIM, int NST, typename TS>
static void launch_patch_tma_ts(const LevelDev& L, const TS* inv, int interior, long long count, const float* r,
                                float* out, int mode, DevStatus* st, cudaStream_t s) {
  using C = TmaCfg<DIM, NST, TS>;
  const long long groups = (count + C::PPI - 1) / C::PPI;
  // the grid is persistent (grid-stride over the patches): every CTA must be resident,
  // so size it by the occupancy the registers and shared memory actually allow
  static int per_sm = -1;
  if (per_sm < 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_tma<DIM, NST, TS>, C::THREADS,
                                                      C::smem_bytes) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    if (per_sm < 1) per_sm = 1;
  }
  const long long cap = 152LL * per_sm;
  const long long grid = groups < cap ? groups : cap;
  if (grid <= 0) return;
  const int early = (!interior && mode == OUT_SCRATCH && L.split && L.nbnd > 0) ? 1 : 0;   // boundary kernel next
  launch_pdl(k_patch_tma<DIM, NST, TS>, (unsigned)grid, C::THREADS, C::smem_bytes, s, L.g, inv,
             interior | (L.split ? 2 : 0), (int)count, r, out, mode, st, L.wait_polls, early);
  count_launch(1);
}

// the level's block-packed inverses: bfloat16 when the level stores them so, else float
template <int DIM, int NST>
static void launch_patch_tma_n(const LevelDev& L, int interior, long long count, const float* r, float* out,
                               int mode, DevStatus* st, cudaStream_t s) {
  if (L.inv16)
    launch_patch_tma_ts<DIM, NST>(L, (const __nv_bfloat16*)L.inv16, interior, count, r, out, mode, st, s);
  else
    launch_patch_tma_ts<DIM, NST>(L, L.inv32, interior, count, r, out, mode, st, s);
}

template <int DIM>
static void launch_patch_variant(int v, const LevelDev& L, int interior, long long count, const float* r, float* out,
                                 int mode, DevStatus* st, cudaStream_t s) {
  if (v == 2) launch_patch_direct<DIM>(L, interior, count, r, out, mode, s);
  else if (v == 1) launch_patch_tma_n<DIM, 3>(L, interior, count, r, out, mode, st, s);
  else launch_patch_tma_n<DIM, 2>(L, interior, count, r, out, mode, st, s);
}

template <int DIM, int NST, typename TS>
static void set_tma_smem_n() {
  cudaFuncSetAttribute(k_patch_tma<DIM, NST, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)TmaCfg<DIM, NST, TS>::smem_bytes);
}

template <int DIM>
static void set_tma_smem() {
  set_tma_smem_n<DIM, 2, float>();
  set_tma_smem_n<DIM, 3, float>();
  set_tma_smem_n<DIM, 2, __nv_bfloat16>();
  set_tma_smem_n<DIM, 3, __nv_bfloat16>();
}

template <int DIM, bool TENSOR, typename R>
static void patch_setup_impl(const LevelDev& L, double gamma, int store32, DevStatus* st, cudaStream_t s) {
  using C = SetupCfg<DIM, TENSOR>;
  const size_t smem = C::smem;
  cudaFuncSetAttribute(k_patch_setup<DIM, TENSOR, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  SetupGeo sg{};
  sg.wdet = 1.0;
  sg.vol = 1.0;
  for (int k = 0; k < 3; ++k) {
    sg.s[k] = k < DIM ? 2.0 / L.g.h[k] : 0.0;
    if (k < DIM) { sg.wdet *= 0.5 * L.g.h[k]; sg.vol *= L.g.h[k]; }
  }
  sg.gvol = gamma / sg.vol;
  R* tab = static_cast<R*>(L.setup_tab);
  k_setup_tables<DIM, R><<<1, 256, 0, s>>>(sg, tab);
  k_patch_setup<DIM, TENSOR, R><<<(unsigned)L.g.nverts, C::THREADS, smem, s>>>(
      L.g, gamma, sg, tab, TENSOR ? L.coef64 : L.mu64, L.inv64, L.pstride, st, L.winv64);
  count_launch(2);
  if (store32) patch_derive32(L, s);
}

template <int DIM, bool TENSOR>
static void patch_setup_arith(const LevelDev& L, double gamma, int store32, int df64, DevStatus* st,
                              cudaStream_t s) {
  if (df64) patch_setup_impl<DIM, TENSOR, DF64>(L, gamma, store32, st, s);
  else patch_setup_impl<DIM, TENSOR, double>(L, gamma, store32, st, s);
}

void patch_setup(const LevelDev& L, double gamma, int store32, int df64, DevStatus* st, cudaStream_t s) {
  if (L.k == 3) {   // FP64 assembly; FP64 (3D mixed: double-float) inversion; FP64 and FP32 copies
    qk_patch_setup(L, gamma, st, s, df64);
    return;
  }
  // shared-memory limit of the FP32 patch kernel, set here, before any graph capture
  if (L.g.dim == 2) set_tma_smem<2>(); else set_tma_smem<3>();
  if (L.g.dim == 2) {
    if (L.tensor) patch_setup_arith<2, true>(L, gamma, store32, df64, st, s);
    else patch_setup_arith<2, false>(L, gamma, store32, df64, st, s);
  } else {
    if (L.tensor) patch_setup_arith<3, true>(L, gamma, store32, df64, st, s);
    else patch_setup_arith<3, false>(L, gamma, store32, df64, st, s);
  }
}

// ---------------------------------------------------------------------------
// FP32 copies of the FP64 inverses (packed by diagonals, every vertex)
// ---------------------------------------------------------------------------
// block-packed (BlockLayout) FP32 copy, one CTA per vertex of inv32 (the interior vertices
// with split storage, else every vertex), entry (i, i+t) of diagonal t rounded to the
// nearest float; padding slots zeroed
__device__ __forceinline__ void store_as(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void store_as(__nv_bfloat16* p, double v) { *p = __double2bfloat16(v); }

template <int DIM, typename TS = float>
__global__ void __launch_bounds__(128) k_derive32(Geom g, int pstride, int split, const double* __restrict__ inv64,
                                                  TS* __restrict__ inv32) {
  constexpr int NP = Sz<DIM>::NP;
  constexpr BlockLayout BL = BlockLayout(NP);
  const long long iv = blockIdx.x;
  long long v = iv;
  if (split) {
    const int nix = g.nv[0] - 2, niy = g.nv[1] - 2;
    const long long vx = iv % nix + 1, q = iv / nix, vy = q % niy + 1, vz = DIM == 3 ? q / niy + 1 : 0;
    v = vx + g.nv[0] * (vy + (long long)g.nv[1] * vz);
  }
  constexpr int OSTRIDE = block_stride<TS>(NP);
  const double* src = inv64 + v * pstride;
  TS* dst = inv32 + iv * OSTRIDE;
  for (int e = 44 * BL.nbp + BL.nbp + (int)threadIdx.x; e < BL.q2; e += blockDim.x) store_as(dst + e, 0.0);
  for (int e = packed_stride(NP) + (int)threadIdx.x; e < OSTRIDE; e += blockDim.x) store_as(dst + e, 0.0);
  for (int t = 0; t < NP; ++t) {
    const int base = diag_start(NP, t);
    for (int i = threadIdx.x; i + t < NP; i += blockDim.x) store_as(dst + BL.index(i, i + t), src[base + i]);
  }
}

// boundary vertices: the free-dof block of the inverse, packed upper triangle by rows,
// rounded to float; one warp per boundary vertex
template <int DIM>
__global__ void __launch_bounds__(256) k_derive32_bnd(Geom g, int pstride, const double* __restrict__ inv64,
                                                      const int* __restrict__ bvid, const long long* __restrict__ boff,
                                                      long long nb, float* __restrict__ bnd32) {
  constexpr int NP = Sz<DIM>::NP;
  const long long b = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nb) return;
  const int v = bvid[b];
  int vx, vy, vz;
  vertex_coords<DIM>(g, v, vx, vy, vz);
  const StarAxes<DIM> ax(g, vx, vy, vz);
  const double* src = inv64 + (long long)v * pstride;
  float* dst = bnd32 + boff[b];
  const int m = ax.m;
  for (int e = lane; e < m * m; e += 32) {
    const int a = e / m, c = e - a * m;
    if (c < a) continue;
    const int i = ax.entry(a), j = ax.entry(c);   // i <= j: entry() increases with the free index
    dst[tri_pos(m, a, c)] = (float)src[diag_start(NP, j - i) + i];
  }
}

void patch_derive32(const LevelDev& L, cudaStream_t s) {
  if (L.k == 3) {   // the FP32 wrapped rows of the order-3 stars
    qk_derive32(L, s);
    return;
  }
  const long long nv32 = L.split ? L.nint : L.g.nverts;
  if (nv32 > 0) {
    if (L.g.dim == 3) k_derive32<3><<<(unsigned)nv32, 128, 0, s>>>(L.g, L.pstride, L.split, L.inv64, L.inv32);
    else k_derive32<2><<<(unsigned)nv32, 128, 0, s>>>(L.g, L.pstride, L.split, L.inv64, L.inv32);
    count_launch(1);
    if (L.inv16) {   // the bfloat16 copy the FP32 cycle streams (ALS_STORE_BF16)
      __nv_bfloat16* d16 = (__nv_bfloat16*)L.inv16;
      if (L.g.dim == 3) k_derive32<3, __nv_bfloat16><<<(unsigned)nv32, 128, 0, s>>>(L.g, L.pstride, L.split, L.inv64, d16);
      else k_derive32<2, __nv_bfloat16><<<(unsigned)nv32, 128, 0, s>>>(L.g, L.pstride, L.split, L.inv64, d16);
      count_launch(1);
    }
  }
  if (L.nbnd > 0) {
    const unsigned blocks = (unsigned)((L.nbnd + 7) / 8);
    if (L.g.dim == 3)
      k_derive32_bnd<3><<<blocks, 256, 0, s>>>(L.g, L.pstride, L.inv64, L.bvid, L.boff, L.nbnd, L.bnd32);
    else
      k_derive32_bnd<2><<<blocks, 256, 0, s>>>(L.g, L.pstride, L.inv64, L.bvid, L.boff, L.nbnd, L.bnd32);
    count_launch(1);
  }
}

int block_stride_bf16(int np) { return block_stride<__nv_bfloat16>(np); }

size_t setup_tab_bytes(int dim) {
  return (size_t)(dim == 2 ? SetupTab<2>::total : SetupTab<3>::total) * sizeof(double);
}

// ---------------------------------------------------------------------------
// K4: y_v = A_v^-1 r|_v, one warp per patch; rows by lanes, diagonals in order
// ---------------------------------------------------------------------------
// y = A r for a symmetric A packed by diagonals, one warp, rows by lanes, over the
// wrapped diagonals t = 0 .. NP-1: row i takes the entry (i, (i + t) mod NP), which is
// entry i of diagonal t while i + t < NP and entry i + t - NP of diagonal NP - t after
// (the symmetric partner), so every (i, j) is used exactly once and every lane of a row
// chunk does useful work at every t (NP^2 products for NP^2 lane-FMAs, where a pass over
// the NP diagonals in both directions would issue 2 NP^2 with half the lanes idle; the FP64
// pipe is this kernel's bound).  Both segments of a wrapped diagonal are contiguous, so the
// loads stay coalesced.
template <typename TF, typename TV, int DIM>
__device__ __forceinline__ void patch_gemv(const TF* __restrict__ S, const TV* rs, int lane, TV (&acc)[(Sz<DIM>::NP + 31) / 32]) {
  constexpr int NP = Sz<DIM>::NP, R = (NP + 31) / 32;
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = TV(0);
#pragma unroll 3
  for (int t = 0; t < NP; ++t) {
    const TF* du = S + diag_start(NP, t);                                 // (i, i + t), i < NP - t
    const TF* dl = S + (t > 0 ? diag_start(NP, NP - t) - (NP - t) : 0);  // (i + t - NP, i), i >= NP - t
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = lane + 32 * k;
      if (i < NP) {
        const int j = i + t;
        const bool up = j < NP;
        acc[k] += (TV)(up ? du[i] : dl[i]) * rs[up ? j : j - NP];
      }
    }
  }
}

template <typename TF, typename TV, int DIM>
__global__ void __launch_bounds__(256) k_patch_apply(Geom g, const TF* __restrict__ inv, int pstride,
                                                     const TV* __restrict__ r, TV* __restrict__ out) {
  constexpr int NP = Sz<DIM>::NP, NB = Sz<DIM>::NB, R = (NP + 31) / 32;
  __shared__ TV rsh[8][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  pdl_wait();
  for (long long v = (long long)blockIdx.x * (blockDim.x >> 5) + w; v < g.nverts; v += nwarps) {
    int vx, vy, vz;
    vertex_coords<DIM>(g, v, vx, vy, vz);
    for (int i = lane; i < NP; i += 32) {
      long long nd;
      const bool ok = patch_node<DIM>(g, vx, vy, vz, i % NB, nd);
      rsh[w][i] = ok ? r[(i / NB) * g.N + nd] : TV(0);
    }
    __syncwarp();
    TV acc[R];
    patch_gemv<TF, TV, DIM>(inv + v * pstride, rsh[w], lane, acc);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = lane + 32 * k;
      if (i < NP) out[patch_out_index<DIM>(g, vx, vy, vz, i)] = acc[k];
    }
    __syncwarp();
  }
}

// z on GX consecutive nodes of a node row = sum of the outputs of the patches whose
// stars contain each node (row layout, patch_out_index): per (y, z) tap pair the
// chunk x = 4j .. 4j+3 reads the six contiguous columns 6j+1 .. 6j+6 (node 4j:
// first; 4j+1: second and third; 4j+2: fourth; 4j+3: fifth and sixth).  Fixed
// order; Dirichlet nodes get 0; divided by den[0] when den is given.
template <typename TV, int DIM>
__device__ __forceinline__ void patch_gather_body(unsigned bx, const Geom& g, const TV* __restrict__ out,
                                                  TV* __restrict__ z, const TV* __restrict__ den) {
  __shared__ TV inv_den;
  pdl_wait();
  if (den) {                        // one division per block, not per entry
    if (threadIdx.x == 0) inv_den = den[0] != TV(0) ? TV(1) / den[0] : TV(0);
    __syncthreads();
  }
  RowChunk rc;
  if (!row_chunk(g, DIM, bx * blockDim.x + threadIdx.x, rc)) return;
  const int nn0 = g.nn[0];
  TV acc[GX];
#pragma unroll
  for (int q = 0; q < GX; ++q) acc[q] = TV(0);
  const bool row_bnd = rc.y == 0 || rc.y == g.nn[1] - 1 || (DIM == 3 && (rc.z == 0 || rc.z == g.nn[2] - 1));
  if (!row_bnd) {
    // per axis: even node 2v -> vertex v (offset 1); odd node 2v+1 -> vertices v (offset 2), v+1 (offset 0)
    int vyv[2], oyv[2], vzv[2], ozv[2];
    bool oky[2], okz[2];
    if (rc.y & 1) { vyv[0] = rc.y >> 1; oyv[0] = 2; vyv[1] = vyv[0] + 1; oyv[1] = 0; oky[0] = oky[1] = true; }
    else { vyv[0] = rc.y >> 1; oyv[0] = 1; oky[0] = true; vyv[1] = 0; oyv[1] = 0; oky[1] = false; }
    if (DIM == 3) {
      if (rc.z & 1) { vzv[0] = rc.z >> 1; ozv[0] = 2; vzv[1] = vzv[0] + 1; ozv[1] = 0; okz[0] = okz[1] = true; }
      else { vzv[0] = rc.z >> 1; ozv[0] = 1; okz[0] = true; vzv[1] = 0; ozv[1] = 0; okz[1] = false; }
    } else {
      vzv[0] = 0; ozv[0] = 0; okz[0] = true; vzv[1] = 0; ozv[1] = 0; okz[1] = false;
    }
    const int ncol = 3 * g.nv[0];
    const int L = DIM == 3 ? 3 : 1;
    const int p0 = 6 * rc.j + 1;
#pragma unroll
    for (int tz = 0; tz < (DIM == 3 ? 2 : 1); ++tz)
#pragma unroll
      for (int ty = 0; ty < 2; ++ty) {
        if (!(oky[ty] && okz[tz])) continue;
        const int row = ((rc.c * L + ozv[tz]) * 3 + oyv[ty]) * (g.nv[1] * g.nv[2]) + vzv[tz] * g.nv[1] + vyv[ty];
        const TV* rowp = out + (long long)row * ncol;
        TV v[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int p = p0 + k;
          v[k] = p < ncol ? rowp[p] : TV(0);
        }
        acc[0] += v[0];
        acc[1] += v[1] + v[2];
        acc[2] += v[3];
        acc[3] += v[4] + v[5];
      }
  }
#pragma unroll
  for (int q = 0; q < GX; ++q) {
    const int xi = GX * rc.j + q;
    if (xi >= nn0) break;
    TV vq = (row_bnd || xi == 0 || xi == nn0 - 1) ? TV(0) : acc[q];
    if (den) vq *= inv_den;
    z[rc.t0 + q] = vq;
  }
}

template <typename TV, int DIM>
__global__ void k_patch_gather(Geom g, const TV* __restrict__ out, TV* __restrict__ z,
                               const TV* __restrict__ den) {
  patch_gather_body<TV, DIM>(blockIdx.x, g, out, z, den);
}

static unsigned row_gather_blocks(const Geom& g, int dim) {
  const long long th = (long long)dim * g.nn[1] * g.nn[2] * ((g.nn[0] + GX - 1) / GX);
  return (unsigned)((th + 255) / 256);
}

size_t patch_scratch_bytes(const LevelDev& L, int prec) {
  return (size_t)L.g.nverts * L.np * (prec == PREC_F64 ? sizeof(double) : sizeof(float));
}

template <typename TF, typename TV, int DIM>
static void smooth_impl(const LevelDev& L, const TF* inv, const void* r, void* z, void* scratch, cudaStream_t s,
                        cudaEvent_t e0, cudaEvent_t e1, const void* den) {
  const long long warps = L.g.nverts;
  const unsigned blocks = (unsigned)std::min<long long>((warps + 7) / 8, 152LL * 16);
  // External records become event-record nodes when the stream is being captured
  if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
  launch_pdl(k_patch_apply<TF, TV, DIM>, blocks, 256, 0, s, L.g, inv, L.pstride, (const TV*)r, (TV*)scratch);
  if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
  launch_pdl(k_patch_gather<TV, DIM>, row_gather_blocks(L.g, DIM), 256, 0, s, L.g, (const TV*)scratch, (TV*)z,
             (const TV*)den);
  count_launch(2);
}

// All star products y_v = A_v^-1 r|_v of a level into the scratch rows (FP32) with kernel
// variant v: the interior stars in the variant's kernel (bracketed by e0/e1 when given),
// then the boundary stars in k_patch_bnd, which runs beside it (see k_patch_bnd).
template <int DIM>
static void star_products(int v, const LevelDev& L, const float* r, float* scratch, cudaStream_t s, cudaEvent_t e0,
                          cudaEvent_t e1) {
  if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
  launch_patch_variant<DIM>(v, L, 0, L.split ? L.nint : L.g.nverts, r, scratch, OUT_SCRATCH, L.status, s);
  if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
  if (L.split) launch_patch_bnd<DIM>(L, r, scratch, s);
}

template <int DIM>
static void smooth_tma(const LevelDev& L, const void* r, void* z, void* scratch, cudaStream_t s, cudaEvent_t e0,
                       cudaEvent_t e1, const void* den) {
  star_products<DIM>(patch_variant(L), L, (const float*)r, (float*)scratch, s, e0, e1);
  launch_pdl(k_patch_gather<float, DIM>, row_gather_blocks(L.g, DIM), 256, 0, s, L.g, (const float*)scratch,
             (float*)z, (const float*)den);
  count_launch(1);
}

void patch_products(const LevelDev& L, const void* r, void* scratch, cudaStream_t s, cudaEvent_t e0,
                    cudaEvent_t e1) {
  if (L.g.dim == 2) star_products<2>(patch_variant(L), L, (const float*)r, (float*)scratch, s, e0, e1);
  else star_products<3>(patch_variant(L), L, (const float*)r, (float*)scratch, s, e0, e1);
}

void patch_smooth(const LevelDev& L, int prec, const void* r, void* z, void* scratch, cudaStream_t s,
                  cudaEvent_t e0, cudaEvent_t e1, const void* den) {
  if (L.k == 3) {
    if (e0) cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);
    qk_patch_smooth(L, prec, r, z, scratch, den, s);
    if (e1) cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
    return;
  }
  if (prec == PREC_F64) {
    if (L.g.dim == 2) smooth_impl<double, double, 2>(L, L.inv64, r, z, scratch, s, e0, e1, den);
    else smooth_impl<double, double, 3>(L, L.inv64, r, z, scratch, s, e0, e1, den);
  } else {
    if (L.g.dim == 2) smooth_tma<2>(L, r, z, scratch, s, e0, e1, den);
    else smooth_tma<3>(L, r, z, scratch, s, e0, e1, den);
  }
}

// ---------------------------------------------------------------------------
// local solves on coarse-cell interiors (robust transfer, Eq. (Ptilde)):
// coarse cell K <-> fine vertex 2K+1, whose star is exactly int(K)
// ---------------------------------------------------------------------------
template <typename TF, typename TV, int DIM>
__global__ void __launch_bounds__(256) k_interior_solve(Geom g, const TF* __restrict__ inv, int pstride,
                                                        const TV* __restrict__ in, TV* __restrict__ out,
                                                        int subtract) {
  constexpr int NP = Sz<DIM>::NP, NB = Sz<DIM>::NB, R = (NP + 31) / 32;
  __shared__ TV rsh[8][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ncx = g.n[0] / 2, ncy = g.n[1] / 2, ncz = DIM == 3 ? g.n[2] / 2 : 1;
  const long long ncoarse = (long long)ncx * ncy * ncz;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  pdl_wait();
  for (long long K = (long long)blockIdx.x * (blockDim.x >> 5) + w; K < ncoarse; K += nwarps) {
    const int kx = (int)(K % ncx), ky = (int)((K / ncx) % ncy), kz = DIM == 3 ? (int)(K / ((long long)ncx * ncy)) : 0;
    const int vx = 2 * kx + 1, vy = 2 * ky + 1, vz = DIM == 3 ? 2 * kz + 1 : 0;
    const long long v = (long long)vx + (long long)g.nv[0] * ((long long)vy + (long long)g.nv[1] * vz);
    for (int i = lane; i < NP; i += 32) {
      long long nd;
      patch_node<DIM>(g, vx, vy, vz, i % NB, nd);  // always interior
      rsh[w][i] = in[(i / NB) * g.N + nd];
    }
    __syncwarp();
    TV acc[R];
    patch_gemv<TF, TV, DIM>(inv + v * pstride, rsh[w], lane, acc);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = lane + 32 * k;
      if (i < NP) {
        long long nd;
        patch_node<DIM>(g, vx, vy, vz, i % NB, nd);
        TV* o = out + (i / NB) * g.N + nd;
        *o = subtract ? *o - acc[k] : acc[k];
      }
    }
    __syncwarp();
  }
}

template <typename TF, typename TV, int DIM>
static void interior_impl(const LevelDev& L, const TF* inv, const void* in, void* out, int subtract, cudaStream_t s) {
  long long nc = (long long)(L.g.n[0] / 2) * (L.g.n[1] / 2) * (DIM == 3 ? L.g.n[2] / 2 : 1);
  if (!subtract) cudaMemsetAsync(out, 0, sizeof(TV) * L.g.N * DIM, s);
  const unsigned blocks = (unsigned)std::min<long long>((nc + 7) / 8, 152LL * 16);
  launch_pdl(k_interior_solve<TF, TV, DIM>, blocks, 256, 0, s, L.g, inv, L.pstride, (const TV*)in, (TV*)out, subtract);
  count_launch(1);
}

void patch_interior_solve(const LevelDev& fine, int prec, const void* in, void* out, int subtract, cudaStream_t s) {
  if (fine.k == 3) {
    qk_interior_solve(fine, prec, in, out, subtract, s);
    return;
  }
  if (prec == PREC_F64) {
    if (fine.g.dim == 2) interior_impl<double, double, 2>(fine, fine.inv64, in, out, subtract, s);
    else interior_impl<double, double, 3>(fine, fine.inv64, in, out, subtract, s);
  } else {
    const long long nc = (long long)(fine.g.n[0] / 2) * (fine.g.n[1] / 2) * (fine.g.dim == 3 ? fine.g.n[2] / 2 : 1);
    if (!subtract) cudaMemsetAsync(out, 0, sizeof(float) * fine.g.N * fine.g.dim, s);
    const int md = subtract ? OUT_SUBTRACT : OUT_WRITE;
    const int v = patch_variant(fine);
    if (fine.g.dim == 2) launch_patch_variant<2>(v, fine, 1, nc, (const float*)in, (float*)out, md, fine.status, s);
    else launch_patch_variant<3>(v, fine, 1, nc, (const float*)in, (float*)out, md, fine.status, s);
  }
}

// ---------------------------------------------------------------------------
// merged launches (batch.cuh): FP32, 2D and 3D instances in one launch.  The
// persistent kernels (TMA ring, direct loads, boundary stars) give every instance a
// share of the launch's blocks in proportion to its star groups, so that the launch
// fills the resident CTAs of the GPU once; within its share an instance's blocks
// stride over its groups exactly as a single-instance launch does over its grid.
// ---------------------------------------------------------------------------
struct PatchArgs {
  Geom g;
  const float* inv;
  int wl, count;
  const float* r;
  float* out;
  int mode;
  DevStatus* st;
  int wait_polls, early;
  // boundary stars
  const float* bnd32;
  const int* bvid;
  const long long* boff;
  long long nb;
  // gather
  const float* den;
};

template <int NST>
__global__ void __launch_bounds__(64) k_patch_tma_b(const __grid_constant__ BatchTab<PatchArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const PatchArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i], gx = tb.start[i + 1] - tb.start[i];
  if (a.g.dim == 3) patch_tma_body<3, NST>(bx, gx, a.g, a.inv, a.wl, a.count, a.r, a.out, a.mode, a.st, a.wait_polls, a.early);
  else patch_tma_body<2, NST>(bx, gx, a.g, a.inv, a.wl, a.count, a.r, a.out, a.mode, a.st, a.wait_polls, a.early);
}
__global__ void __launch_bounds__(128) k_patch_direct_b(const __grid_constant__ BatchTab<PatchArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const PatchArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i], gx = tb.start[i + 1] - tb.start[i];
  if (a.g.dim == 3) patch_direct_body<3>(bx, gx, a.g, a.inv, a.wl, a.count, a.r, a.out, a.mode);
  else patch_direct_body<2>(bx, gx, a.g, a.inv, a.wl, a.count, a.r, a.out, a.mode);
}
__global__ void __launch_bounds__(256) k_patch_bnd_b(const __grid_constant__ BatchTab<PatchArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const PatchArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i], gx = tb.start[i + 1] - tb.start[i];
  if (a.g.dim == 3) patch_bnd_body<3>(bx, gx, a.g, a.bnd32, a.bvid, a.boff, a.nb, a.r, a.out);
  else patch_bnd_body<2>(bx, gx, a.g, a.bnd32, a.bvid, a.boff, a.nb, a.r, a.out);
}
__global__ void __launch_bounds__(256) k_patch_gather_b(const __grid_constant__ BatchTab<PatchArgs> tb) {
  const int i = batch_slot(tb, blockIdx.x);
  const PatchArgs& a = tb.a[i];
  const unsigned bx = blockIdx.x - tb.start[i];
  if (a.g.dim == 3) patch_gather_body<float, 3>(bx, a.g, a.r, a.out, a.den);
  else patch_gather_body<float, 2>(bx, a.g, a.r, a.out, a.den);
}

template <int NST>
static size_t tma_b_smem() {
  return std::max(TmaCfg<2, NST>::smem_bytes, TmaCfg<3, NST>::smem_bytes);
}

// resident CTAs per SM of a merged patch kernel (variant 0, 1: TMA ring; 2: direct; 3: boundary)
static int batch_per_sm(int variant) {
  static int cache[4] = {-1, -1, -1, -1};
  if (cache[variant] >= 0) return cache[variant];
  int v = 0;
  cudaError_t e = cudaSuccess;
  if (variant == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_patch_tma_b<2>, 64, tma_b_smem<2>());
  else if (variant == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_patch_tma_b<3>, 64, tma_b_smem<3>());
  else if (variant == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_patch_direct_b, 128, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_patch_bnd_b, 256, 0);
  if (e != cudaSuccess) { cudaGetLastError(); v = 1; }
  cache[variant] = v < 1 ? 1 : v;
  return cache[variant];
}
int batch_patch_occupancy(int variant) { return batch_per_sm(variant); }

// shared-memory opt-in of the merged TMA-ring kernels (before any capture)
void batch_patch_prepare() {
  cudaFuncSetAttribute(k_patch_tma_b<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_b_smem<2>());
  cudaFuncSetAttribute(k_patch_tma_b<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_b_smem<3>());
  for (int v = 0; v < 4; ++v) batch_per_sm(v);
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
  }
  return n;
}

// stars per iteration of a variant's CTA for an instance of dimension dim
static int stars_per_group(int variant, int dim) {
  if (variant == 2) return dim == 3 ? DirCfg<3>::PPC : DirCfg<2>::PPC;
  return dim == 3 ? TmaCfg<3, 2>::PPI : TmaCfg<2, 2>::PPI;
}

// one merged launch of a variant's kernel over (item, wl, count, mode); early: the
// boundary-star launch follows
static int launch_patch_b(int variant, const std::vector<PatchArgs>& a, cudaStream_t s) {
  std::vector<long long> work;
  for (const PatchArgs& x : a) {
    const int ppg = stars_per_group(variant, x.g.dim);
    work.push_back(((long long)x.count + ppg - 1) / ppg);
  }
  const long long per_sm = batch_per_sm(variant);
  const long long cap = (long long)sm_count() * (variant == 2 ? 8 : per_sm);
  const std::vector<unsigned> nb = persistent_shares(work, (long long)sm_count() * per_sm, cap);
  if (variant == 2) return launch_batch(k_patch_direct_b, a, nb, 128, 0, s);
  if (variant == 1) return launch_batch(k_patch_tma_b<3>, a, nb, 64, tma_b_smem<3>(), s);
  return launch_batch(k_patch_tma_b<2>, a, nb, 64, tma_b_smem<2>(), s);
}

static PatchArgs patch_args(const LevelDev& L, int wl, long long count, const void* r, void* out, int mode) {
  PatchArgs a{};
  a.g = L.g;
  a.inv = L.inv32;
  a.wl = wl | (L.split ? 2 : 0);
  a.count = (int)count;
  a.r = (const float*)r;
  a.out = (float*)out;
  a.mode = mode;
  a.st = L.status;
  a.wait_polls = L.wait_polls;
  a.bnd32 = L.bnd32;
  a.bvid = L.bvid;
  a.boff = L.boff;
  a.nb = L.nbnd;
  return a;
}

int batch_star_products(int variant, const std::vector<BPatch>& items, cudaStream_t s) {
  std::vector<PatchArgs> a, bnd;
  std::vector<long long> bwork;
  for (const BPatch& it : items) {
    const LevelDev& L = *it.L;
    a.push_back(patch_args(L, 0, L.split ? L.nint : L.g.nverts, it.r, it.out, OUT_SCRATCH));
    if (L.split && L.nbnd > 0) {
      bnd.push_back(a.back());
      bwork.push_back((L.nbnd + 7) / 8);
    }
  }
  // the TMA-ring kernel lets the boundary-star kernel start once its dependency wait returned
  if (variant != 2 && !bnd.empty())
    for (PatchArgs& x : a) x.early = 1;
  int n = launch_patch_b(variant, a, s);
  if (!bnd.empty()) {
    const std::vector<unsigned> nb = persistent_shares(bwork, (long long)sm_count() * batch_per_sm(3), 152LL * 16);
    n += launch_batch(k_patch_bnd_b, bnd, nb, 256, 0, s);
  }
  count_launch(n);
  return n;
}

int batch_patch_gather(const std::vector<BPatch>& items, cudaStream_t s) {
  std::vector<PatchArgs> a;
  std::vector<unsigned> nb;
  for (const BPatch& it : items) {
    PatchArgs x{};
    x.g = it.L->g;
    x.r = (const float*)it.out;   // the scratch rows of the star products
    x.out = (float*)it.z;
    x.den = (const float*)it.den;
    a.push_back(x);
    nb.push_back(row_gather_blocks(it.L->g, it.L->g.dim));
  }
  const int n = launch_batch(k_patch_gather_b, a, nb, 256, 0, s);
  count_launch(n);
  return n;
}

int batch_interior_solve(int variant, const std::vector<BPatch>& items, int subtract, cudaStream_t s) {
  std::vector<PatchArgs> a;
  std::vector<BZero> z;
  for (const BPatch& it : items) {
    const Geom& g = it.L->g;
    const long long nc = (long long)(g.n[0] / 2) * (g.n[1] / 2) * (g.dim == 3 ? g.n[2] / 2 : 1);
    a.push_back(patch_args(*it.L, 1, nc, it.r, it.out, subtract ? OUT_SUBTRACT : OUT_WRITE));
    if (!subtract) z.push_back(BZero{it.out, g.N * g.dim});
  }
  int n = 0;
  if (!z.empty()) n += batch_zero(z, s);   // counted there
  const int m = launch_patch_b(variant, a, s);
  count_launch(m);
  return n + m;
}

// Autotuner: times each FP32 patch-kernel variant on this level (one warm-up and
// three timed launches each, CUDA events on the stream, r and scratch supplied
// by the caller) and stores the fastest in L.patch_kernel.  Runs outside any
// stream capture; waits for its own work.  Returns the chosen variant.
int patch_autotune(LevelDev& L, const void* r, void* scratch, cudaStream_t s, float* ms_out) {
  const long long launches0 = launch_count();
  if (L.k == 3) { L.patch_kernel = 0; return 0; }   // one star kernel at order 3
  if (forced_patch_kernel() >= 0) { L.patch_kernel = forced_patch_kernel(); return L.patch_kernel; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = 0;
  float best_ms = 1e30f;
  for (int v = 0; v < 3; ++v) {
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) cudaEventRecord(e0, s);
      if (L.g.dim == 2) star_products<2>(v, L, (const float*)r, (float*)scratch, s, nullptr, nullptr);
      else star_products<3>(v, L, (const float*)r, (float*)scratch, s, nullptr, nullptr);
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) ms_out[v] = ms / 3.f;
    if (ms < best_ms) { best_ms = ms; best = v; }
  }
  count_launch(-(launch_count() - launches0));   // tuning launches are not work of the caller's step
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.patch_kernel = best;
  return best;
}

}  // namespace als
