// Allocation-free variant of the vertex-star smoother apply.
//
// Who this is for: code that must not allocate device memory at the moment it
// smooths -- a hard real-time loop that has budgeted all device memory in
// advance, a plugin whose host framework owns the allocator and forbids direct
// cudaMalloc, or a caller on a path where the implicit device synchronisation of
// an allocation is not acceptable.  Such callers hold the patch inverses and the
// vectors already; what they cannot provide is the per-patch scratch buffer (one
// d*3^d vector per vertex) that the two-step, deterministic smoother needs
// between its patch kernel and its gather kernel.
//
// This file keeps that scratch in one file-scope device array of fixed size
// (ALS_STATIC_SCRATCH_BYTES).  Every GPU that loads the library reserves it
// until the process exits.  All calls share it, so calls that overlap on the
// GPU (different streams, or different host threads) race and give wrong
// results; serialise them.  Every scratch entry a call reads is written
// earlier in the same call, so nothing has to start at zero.
#include <cuda_runtime.h>

#include <atomic>

#include "../../include/alstokes.h"
#include "common.cuh"

namespace als {
namespace {

static __device__ __align__(256) unsigned char g_star_scratch[ALS_STATIC_SCRATCH_BYTES];

// Per device, looked up once by the first call made with that device current: the
// device address of g_star_scratch (in host code the symbol itself is only a host-side
// stand-in) and the SM count that sizes the patch kernel's grid.  Atomic, because
// host threads may call concurrently; a cudaDeviceReset reloads the module, after
// which these values are stale (the call is not meant to outlive the context).
constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_addr[kMaxDevices];
std::atomic<int> g_sm_count[kMaxDevices];

template <int DIM>
__device__ __forceinline__ bool star_node(const Geom& g, int vx, int vy, int vz, int o, long long& nd) {
  const int i = 2 * vx + o % 3 - 1;
  const int j = 2 * vy + (o / 3) % 3 - 1;
  const int k = (DIM == 3) ? 2 * vz + o / 9 - 1 : 0;
  if (i <= 0 || i >= g.nn[0] - 1 || j <= 0 || j >= g.nn[1] - 1) return false;
  if (DIM == 3 && (k <= 0 || k >= g.nn[2] - 1)) return false;
  nd = node_id(g, i, j, k);
  return true;
}

// y_v = A_v^-1 r|_v for every vertex v (one warp per patch), into the static scratch
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_star_static(Geom g, const T* __restrict__ inv, int pstride,
                                                     const T* __restrict__ r, T* __restrict__ out) {
  constexpr int NP = Sz<DIM>::NP, NB = Sz<DIM>::NB, R = (NP + 31) / 32;
  __shared__ T rsh[8][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long v = (long long)blockIdx.x * (blockDim.x >> 5) + w; v < g.nverts; v += nwarps) {
    const int vx = (int)(v % g.nv[0]);
    const int vy = (int)((v / g.nv[0]) % g.nv[1]);
    const int vz = DIM == 3 ? (int)(v / ((long long)g.nv[0] * g.nv[1])) : 0;
    for (int i = lane; i < NP; i += 32) {
      long long nd;
      rsh[w][i] = star_node<DIM>(g, vx, vy, vz, i % NB, nd) ? r[(i / NB) * g.N + nd] : T(0);
    }
    __syncwarp();
    T acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = T(0);
    const T* S = inv + v * pstride;
    for (int t = 0; t < NP; ++t) {
      const T* d = S + diag_start(NP, t);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const int i = lane + 32 * k;
        if (i < NP) {
          if (i + t < NP) acc[k] += d[i] * rsh[w][i + t];
          if (t > 0 && i >= t) acc[k] += d[i - t] * rsh[w][i - t];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int i = lane + 32 * k;
      if (i < NP) out[v * NP + i] = acc[k];
    }
    __syncwarp();
  }
}

// z(node) = sum of the scratch values of the patches containing the node, fixed order
template <typename T, int DIM>
__global__ void k_star_static_gather(Geom g, const T* __restrict__ out, T* __restrict__ z) {
  constexpr int NP = Sz<DIM>::NP, NB = Sz<DIM>::NB;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.N * DIM) return;
  const int c = (int)(t / g.N);
  const long long nd = t % g.N;
  const int idx[3] = {(int)(nd % g.nn[0]), (int)((nd / g.nn[0]) % g.nn[1]), (int)(nd / ((long long)g.nn[0] * g.nn[1]))};
  if (on_boundary(g, idx[0], idx[1], idx[2])) { z[t] = T(0); return; }
  int nva[3] = {1, 1, 1}, vv[3][2] = {{0, 0}, {0, 0}, {0, 0}}, oo[3][2] = {{1, 1}, {1, 1}, {1, 1}};
  for (int a = 0; a < DIM; ++a) {
    if ((idx[a] & 1) == 0) { vv[a][0] = idx[a] >> 1; oo[a][0] = 1; }
    else { nva[a] = 2; vv[a][0] = (idx[a] - 1) >> 1; oo[a][0] = 2; vv[a][1] = (idx[a] + 1) >> 1; oo[a][1] = 0; }
  }
  T acc = T(0);
  for (int cz = 0; cz < nva[2]; ++cz)
    for (int cy = 0; cy < nva[1]; ++cy)
      for (int cx = 0; cx < nva[0]; ++cx) {
        const long long vid = (long long)vv[0][cx] + (long long)g.nv[0] * ((long long)vv[1][cy] +
                              (DIM == 3 ? (long long)g.nv[1] * vv[2][cz] : 0));
        const int o = oo[0][cx] + 3 * oo[1][cy] + (DIM == 3 ? 9 * oo[2][cz] : 0);
        acc += out[vid * NP + c * NB + o];
      }
  z[t] = acc;
}

template <typename T, int DIM>
cudaError_t launch(Geom g, const void* inv, const void* r, void* z, void* scratch, int sms, cudaStream_t s) {
  const long long blocks = (g.nverts + 7) / 8;
  const long long cap = 16LL * sms;
  int pstride = packed_stride(Sz<DIM>::NP);
  const T* inv_t = (const T*)inv;
  const T* r_t = (const T*)r;
  T* out_t = (T*)scratch;
  T* z_t = (T*)z;
  void* a1[] = {&g, &inv_t, &pstride, &r_t, &out_t};
  cudaError_t e = cudaLaunchKernel((const void*)k_star_static<T, DIM>, dim3((unsigned)(blocks < cap ? blocks : cap)),
                                   dim3(256), a1, 0, s);
  if (e != cudaSuccess) return e;
  const long long tot = g.N * DIM;
  const T* sc_t = (const T*)scratch;
  void* a2[] = {&g, &sc_t, &z_t};
  return cudaLaunchKernel((const void*)k_star_static_gather<T, DIM>, dim3((unsigned)((tot + 255) / 256)), dim3(256),
                          a2, 0, s);
}

}  // namespace
}  // namespace als

extern "C" als_status als_star_smooth_static(int dim, const int* n, int prec, const void* inv, const void* r,
                                             void* z, void* stream) {
  using namespace als;
  if ((dim != 2 && dim != 3) || !n || !inv || !r || !z) return ALS_EINVAL;
  if (prec != ALS_PREC_FP64 && prec != ALS_PREC_FP32) return ALS_EINVAL;
  // every axis is bounded before any product is formed, so none of them can wrap
  constexpr int kMaxCells = 4096;
  for (int k = 0; k < dim; ++k)
    if (n[k] < 1 || n[k] > kMaxCells) return ALS_EINVAL;
  Geom g{};
  g.dim = dim;
  for (int k = 0; k < 3; ++k) {
    const bool act = k < dim;
    g.n[k] = act ? n[k] : 1;
    g.nn[k] = act ? 2 * n[k] + 1 : 1;
    g.nv[k] = act ? n[k] + 1 : 1;
    g.h[k] = act ? 1.0 / n[k] : 0.0;
  }
  g.N = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  g.ncells = (long long)g.n[0] * g.n[1] * g.n[2];
  g.nverts = (long long)g.nv[0] * g.nv[1] * g.nv[2];
  const long long np = dim == 2 ? 18 : 81;
  const long long need = g.nverts * np * (prec == ALS_PREC_FP64 ? 8 : 4);   // < 4097^3 * 648, no overflow
  if (need > (long long)ALS_STATIC_SCRATCH_BYTES) return ALS_EINVAL;  // mesh too large for the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ALS_ECUDA;
  void* scratch = g_scratch_addr[dev].load();
  int sms = g_sm_count[dev].load();
  if (!scratch || sms <= 0) {
    // set-up of this device: the array's device address and the SM count
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_star_scratch) != cudaSuccess || !p) return ALS_ECUDA;
    int count = 0;
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count <= 0)
      return ALS_ECUDA;
    g_scratch_addr[dev].store(p);
    g_sm_count[dev].store(count);
    scratch = p;
    sms = count;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (prec == ALS_PREC_FP64) {
    e = dim == 2 ? launch<double, 2>(g, inv, r, z, scratch, sms, s) : launch<double, 3>(g, inv, r, z, scratch, sms, s);
  } else {
    e = dim == 2 ? launch<float, 2>(g, inv, r, z, scratch, sms, s) : launch<float, 3>(g, inv, r, z, scratch, sms, s);
  }
  return e == cudaSuccess ? ALS_OK : ALS_ECUDA;
}
