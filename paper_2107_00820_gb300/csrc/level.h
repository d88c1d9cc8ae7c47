// Host-side description of one multigrid level as seen by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "reduce.cuh"

namespace als {

// Poll limit of the bounded mbarrier waits in the FP32 star-smoother kernel (each
// poll backs off ~256 ns, so the default gives up after well over a second).
constexpr int kWaitPolls = 1 << 22;

struct LevelDev {
  Geom g;
  int k = 2;             // polynomial order of the velocity: 2 ([Q2]^d x P1disc) or 3 ([Q3]^d x P2disc, qk.cu, qk3.cu)
  int npr = 0;           // pressure unknowns per cell (d + 1, or 6 / 10 at order 3 in 2D / 3D)
  int nq = 0;            // Gauss points per cell ((k + 1)^d)
  int tensor;            // 0: scalar mu per point, 1: Mandel tensor per point
  int ncoef;             // values per point (1 or NC)
  double* coef64;        // [cell][3^d][ncoef]
  float* coef32;
  double* mu64;          // scalar viscosity per point (mu or mu_eff), FP64
  // vertex-star patch inverses: FP64 packed symmetric by diagonals, one per vertex
  // (identity rows at absent and Dirichlet nodes); FP32 block-packed (BlockLayout) for
  // every vertex, or, with split storage (large levels), for the interior vertices only
  // (1 <= v_k <= n_k - 1, interior index x-fastest) and a compact FP32 copy of each
  // boundary vertex's star restricted to its free dofs
  double* inv64;
  float* inv32;
  // ALS_STORE_BF16: the same block-packed stars as inv32 rounded to bfloat16 (stride
  // rounded to 8 entries), which the FP32 star kernels then stream instead; NULL otherwise
  void* inv16 = nullptr;
  int split;             // split storage (see above)
  float* bnd32;          // boundary stars: packed upper triangle by rows, m x m, m = free dofs
  int* bvid;             // boundary vertex ids (nbnd), ascending
  long long* boff;       // offset of each boundary star's compact inverse in bnd32
  long long nint;        // interior vertices, prod(n_k - 1)
  long long nbnd;        // boundary vertices, nverts - nint
  int np;                // patch size d*3^d
  int pstride;           // entries per patch (padded)
  DevStatus* status;     // where kernels of this level record device-side failures
  void* ebuf;            // per-cell output buffer of the operator apply, [cell][d][3^d] (FP64-sized)
  // W^-1 of the augmentation when W = M_p(1/mu): per-cell (d+1)^2 blocks; NULL when W = M_p
  double* winv64;
  float* winv32;
  int patch_kernel;      // FP32 patch-kernel variant picked by patch_autotune (-1: not yet tuned)
  float tune_ms[3];      // measured time per launch of each variant (ms)
  void* setup_tab;       // reference tables of the patch setup (setup_tab_bytes)
  int wait_polls = kWaitPolls;   // poll limit of the smoother kernel's pipeline waits
  // order 3 in 3D: workspace of the star setup (qk3_setup_ws_doubles(qk_ws_ctas) doubles,
  // shared by the levels, whose setups run one after another on the context's stream)
  double* qk_ws = nullptr;
  int qk_ws_ctas = 0;
};

enum Prec { PREC_F64 = 0, PREC_F32 = 1 };

// Process-wide count of kernels this library has put on a stream (graph
// replays add the number of kernel nodes of the graph).  Launchers call
// count_launch(); while a V-cycle is being captured the count is attributed
// to the graph instead.
long long launch_count();
void count_launch(long long n);

// ---- operator.cu
void op_apply(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y,
              const void* p_in, void* p_out, cudaStream_t s);
// A_gamma apply (viscous + AL) fused with the reduction that consumes y:
//   y = b + sigma A x (b NULL: y = sigma A x);
//   start = 0: out[j] = (V_j . y) / hn[j] for j < k (k <= KMAXB; Arnoldi dots)
//   start = 1: |y|^2 starts the GMRES cycle st
// out and the GMRES state hold elements of the apply's precision.
struct ApplyEpi {
  const void* b;
  double sigma;
  int k;
  const void* V;
  long long ld;
  void* out;
  int start;
  GmresDev st;
  double* partial;
  // FP32, 3D: when pout is set, the apply's input x is not read but formed from the
  // star-patch outputs pout (row layout) divided by the device scalar pden, and stored
  // into x (the patch gather fused into the cell kernel)
  const void* pout = nullptr;
  const void* pden = nullptr;
};
// e0/e1 (optional) are recorded immediately before and after the cell kernel
void op_apply_epi(const LevelDev& L, int prec, double gamma, const void* x, void* y, const ApplyEpi& e,
                  cudaStream_t s, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);
void op_load_vector(const LevelDev& L, const double* f_qp, double* F, cudaStream_t s);
void op_apply_multi(const LevelDev& L, double gamma, const double* X, double* Y, int nvec,
                    long long stride, cudaStream_t s);

// ---- patches.cu
// df64: assemble and invert in double-float arithmetic (FP32 pairs, about 48 bits),
// enough for the FP32 inverse of the mixed cycle; otherwise in FP64.  L.setup_tab
// holds setup_tab_bytes(dim) bytes of scratch for the level's reference tables.
void patch_setup(const LevelDev& L, double gamma, int store32, int df64, DevStatus* st, cudaStream_t s);
size_t setup_tab_bytes(int dim);
// entries per star of the bfloat16 block-packed copy (inv16)
int block_stride_bf16(int np);
// the FP32 block-packed inverses (inv32) of every patch from the FP64 ones (inv64);
// the setup calls it, and so does the loading of caller-supplied FP64 inverses
void patch_derive32(const LevelDev& L, cudaStream_t s);
// e0/e1 (optional) are recorded immediately before and after the patch kernel
// den (optional device scalar of precision prec): z = D^-1 r / den (0 where den == 0)
void patch_smooth(const LevelDev& L, int prec, const void* r, void* z, void* scratch, cudaStream_t s,
                  cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr, const void* den = nullptr);
size_t patch_scratch_bytes(const LevelDev& L, int prec);
// FP32: the star-patch products y_v = A_v^-1 r|_v into the scratch rows only (their
// node sums are formed by the consumer, see ApplyEpi::pout)
void patch_products(const LevelDev& L, const void* r, void* scratch, cudaStream_t s, cudaEvent_t e0 = nullptr,
                    cudaEvent_t e1 = nullptr);
// times the FP32 patch-kernel variants on this level and keeps the fastest (ms_out[3], optional)
int patch_autotune(LevelDev& L, const void* r, void* scratch, cudaStream_t s, float* ms_out = nullptr);
// local solves on the coarse-cell interiors (stars of the fine vertices at the
// coarse-cell centres):  mode 0: out = sum_K E_K A_K^-1 E_K^T in  (out zeroed first)
//                        mode 1: out -= sum_K E_K A_K^-1 E_K^T in
void patch_interior_solve(const LevelDev& fine, int prec, const void* in, void* out, int subtract,
                          cudaStream_t s);

// ---- qk.cu: the order-3 discretisation ([Q3]^d x P2disc); the dispatchers of
// operator.cu, patches.cu, transfer.cu and coarse.cu call these when L.k == 3, and they
// pass 3D levels on to qk3.cu's qk3_* functions of the same arguments
void qk_tables();
void qk_apply(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y, const void* p_in, void* p_out,
              cudaStream_t s);
void qk_load_vector(const LevelDev& L, const double* f_qp, double* F, cudaStream_t s);
// op_apply_epi at order 3 (the GMRES smoother's Arnoldi step)
void qk_apply_epi(const LevelDev& L, int prec, double gamma, const void* x, void* y, const ApplyEpi& e,
                  cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1);
// per-cell W^-1 (w_mu: W = M_p(1/mu), else M_p) into winv64/winv32 and, if S, the Schur blocks
// of Eq. (P1P2) (variant 0: P1, 1: P2)
void qk_mass_setup(const LevelDev& L, double gamma, int w_mu, int variant, double* winv64, float* winv32, double* S,
                   DevStatus* st, cudaStream_t s);
// df64: 3D levels eliminate in double-float (2D order 3 is FP64 throughout)
void qk_patch_setup(const LevelDev& L, double gamma, DevStatus* st, cudaStream_t s, int df64);
// FP32 entries per star of an order-3 level (inv32 holds the stars in wrapped rows), and
// inv32 formed from inv64
size_t qk_star32_floats(int dim);
void qk_derive32(const LevelDev& L, cudaStream_t s);
void qk_patch_smooth(const LevelDev& L, int prec, const void* r, void* z, void* scratch, const void* den,
                     cudaStream_t s);
void qk_interior_solve(const LevelDev& fine, int prec, const void* in, void* out, int subtract, cudaStream_t s);
void qk_prolong(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf, cudaStream_t s,
                void* xadd);
void qk_restrict(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc, cudaStream_t s,
                 const void* sub);
// ---- qk3.cu: [Q3]^3 x P2disc
void qk3_tables();
void qk3_apply(const LevelDev& L, int prec, int mode, double gamma, const void* x, void* y, const void* p_in,
               void* p_out, cudaStream_t s);
void qk3_load_vector(const LevelDev& L, const double* f_qp, double* F, cudaStream_t s);
void qk3_apply_epi(const LevelDev& L, int prec, double gamma, const void* x, void* y, const ApplyEpi& e,
                   cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1);
void qk3_mass_setup(const LevelDev& L, double gamma, int w_mu, int variant, double* winv64, float* winv32, double* S,
                    DevStatus* st, cudaStream_t s);
// the star setup's CTAs for a level of nverts vertices, and the workspace they need
// (doubles; one 375 x 376 FP64 star matrix per CTA), held in LevelDev::qk_ws
int qk3_setup_ctas(long long nverts);
size_t qk3_setup_ws_doubles(int ctas);
// FP32 entries per star of a 3D order-3 level (inv32 holds the stars in wrapped rows), and
// inv32 formed from inv64
size_t qk3_star32_floats();
void qk3_derive32(const LevelDev& L, cudaStream_t s);
// df64: the elimination in double-float arithmetic (the assembly stays FP64)
void qk3_patch_setup(const LevelDev& L, double gamma, DevStatus* st, cudaStream_t s, int df64);
void qk3_patch_smooth(const LevelDev& L, int prec, const void* r, void* z, void* scratch, const void* den,
                      cudaStream_t s);
void qk3_interior_solve(const LevelDev& fine, int prec, const void* in, void* out, int subtract, cudaStream_t s);
void qk3_prolong(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf, cudaStream_t s,
                 void* xadd);
void qk3_restrict(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc, cudaStream_t s,
                  const void* sub);

// ---- newton.cu
// Coefficients of the Newton linearisation at the finest-level velocity u, at the Gauss
// points of `level` ([cell][3^d] mu, and [cell][3^d][6|21] Mandel C unless C is NULL)
void newton_coeffs(const Geom& fine, const Geom& level, const double* u, double mu_ref, double tau_y, double* C,
                   double* mu, cudaStream_t s);

// ---- transfer.cu
// xf = P_H xc; if xadd, also xadd += P_H xc
void prolong_std(const LevelDev& coarse, const LevelDev& fine, int prec, const void* xc, void* xf,
                 cudaStream_t s, void* xadd = nullptr);
// rc = P_H^T rf, or P_H^T (rf - sub) when sub is given
void restrict_std(const LevelDev& coarse, const LevelDev& fine, int prec, const void* rf, void* rc,
                  cudaStream_t s, const void* sub = nullptr);

// ---- krylov.cu (vector kernels)
void vec_axpby(int prec, long long n, double a, const void* x, double b, void* y, cudaStream_t s);
void vec_axpy_dev(int prec, long long n, const double* a, double sign, const void* x, void* y,
                  cudaStream_t s);
void vec_cast(long long n, const void* src, int src_prec, void* dst, int dst_prec, cudaStream_t s);
void vec_zero(int prec, long long n, void* x, cudaStream_t s);
// out[j] = <V_j, w> for j < k, V stored as k rows of length n with leading dim ld
void vec_multidot(int prec, long long n, int k, const void* V, long long ld, const void* w,
                  double* out, double* partial, cudaStream_t s);
// w -= sum_j V_j h[j]
void vec_multiaxpy(int prec, long long n, int k, const void* V, long long ld, const double* h,
                   void* w, cudaStream_t s);
// y = x * num / den (num, den device scalars, NULL = 1; den <- sqrt(den) if sqrt_den)
void vec_scale_dev(int prec, long long n, const double* num, const double* den, const void* x, void* y,
                   cudaStream_t s, int sqrt_den = 0);
// w <- w + sign * sum_j V_j h_j and nrm2 = |w|^2, one launch
void vec_multiaxpy_norm(int prec, long long n, int k, const void* V, long long ld, const double* h, double sign,
                        void* w, double* partial, double* nrm2, cudaStream_t s);
// GMRES(s) smoother with an unnormalised stored basis (GmresDev): V0 = b and start;
// orthogonalise column j+1 and take the Givens step j; x (+)= Z y and, if t, the
// GMRES residual t = r0 - A Z y from the Arnoldi relation.  s <= KMAXB.
size_t gmres_partial_doubles(long long n);   // workspace of op_apply_epi and gm_* for n entries
void gm_start(int prec, long long n, const void* b, void* V0, double* partial, const GmresDev& st, cudaStream_t s);
void gm_orth(int prec, long long n, int j, const void* V, long long ld, double* partial, const GmresDev& st,
             cudaStream_t s);
void gm_update(int prec, long long n, int k, const void* Z, const void* V, long long ld, const GmresDev& st,
               void* x, int x_zero, void* t, cudaStream_t s);
size_t multidot_partial_doubles(int k);

// ---- merged launches over the instances of a batch (batch.cuh).  FP32, order 2, scalar
// viscosity.  Each call runs one level operation for every item, in one launch per kernel
// the single-instance operation uses (plus one per kBatchMax items beyond the first
// kBatchMax), with each item's arithmetic exactly that of the single-instance call named
// beside it.  Every call returns the number of launches it made.
struct BApply {            // op_apply_epi (e used), or op_apply(OP_AL) (e ignored)
  const LevelDev* L;
  double gamma;
  const void* x;
  void* y;
  ApplyEpi e;
};
int batch_apply_epi(const std::vector<BApply>& items, cudaStream_t s);
int batch_apply_al(const std::vector<BApply>& items, cudaStream_t s);
struct BPatch {            // star products of the smoother (r -> scratch rows), or the local
  const LevelDev* L;       // solves on the coarse-cell interiors (r = in, out)
  const void* r;
  void* out;
  const void* den;         // the gather's divisor (batch_patch_gather), may be NULL
  void* z;                 // the gather's output (batch_patch_gather)
};
// variant: the patch-kernel variant of patch_autotune (0 = TMA ring, 2 stages; 1 = 3 stages;
// 2 = direct loads); every item's interior stars run in it
int batch_star_products(int variant, const std::vector<BPatch>& items, cudaStream_t s);      // patch_products
int batch_patch_gather(const std::vector<BPatch>& items, cudaStream_t s);   // the node sums of patch_smooth
int batch_interior_solve(int variant, const std::vector<BPatch>& items, int subtract, cudaStream_t s);
struct BTransfer {
  const LevelDev* coarse;
  const LevelDev* fine;
  const void* in;
  void* out;
  const void* aux;         // prolong: xadd (out added to it, may be NULL); restrict: sub (may be NULL)
};
int batch_prolong(const std::vector<BTransfer>& items, cudaStream_t s);     // prolong_std
int batch_restrict(const std::vector<BTransfer>& items, cudaStream_t s);    // restrict_std
struct BGmres {            // gm_start (b, V), gm_orth (V, j), gm_update (Z, V, x, t, x_zero)
  long long n;
  const void* b;
  const void* Z;
  void* V;
  long long ld;
  int j;
  double* partial;
  GmresDev st;
  void* x;
  int x_zero;
  void* t;
};
int batch_gm_start(const std::vector<BGmres>& items, cudaStream_t s);
int batch_gm_orth(const std::vector<BGmres>& items, cudaStream_t s);
int batch_gm_update(const std::vector<BGmres>& items, cudaStream_t s);
struct BZero {
  void* x;
  long long n;             // floats
};
int batch_zero(const std::vector<BZero>& items, cudaStream_t s);
// resident CTAs per SM of a merged star kernel (variant 0, 1, 2 as above; 3: boundary stars)
int batch_patch_occupancy(int variant);
// shared-memory opt-ins of the merged star kernels; call before the first capture
void batch_patch_prepare();

}  // namespace als
