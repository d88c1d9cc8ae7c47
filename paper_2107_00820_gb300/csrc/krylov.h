// Device-side Krylov helpers shared by the V-cycle smoother and the outer FGMRES.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace als {

void vec_multiaxpy(int prec, long long n, int k, const void* V, long long ld, const double* h, void* w,
                   cudaStream_t s, double sign);
void dev_sqrt(const double* in, double* out, cudaStream_t s);
void dev_hess_finish(int k, double* hcol, const double* h2, const double* nrm2, cudaStream_t s);
void dev_givens_step(int k, double* H, int ldh, double* cs, double* sn, double* g, double* res, cudaStream_t s);
void dev_hess_givens(int k, double* H, int ldh, const double* h2, const double* nrm2, double* cs, double* sn,
                     double* g, double* res, cudaStream_t s);
void dev_backsolve(int k, const double* H, int ldh, const double* g, double* y, cudaStream_t s);
void dev_init_g(int m, const double* nrm2, double* g, double* beta, cudaStream_t s);
void schur_apply(long long ncells, int npr, const double* S, const double* t, double* z, cudaStream_t s);
void project_constant(long long ncells, int npr, double* p, double* partial, cudaStream_t s);
// atomic minimum of the positive entries of x into *out_bits (the bits of a double; start at +inf)
void vec_min_positive(long long n, const double* x, unsigned long long* out_bits, cudaStream_t s);

// coarse.cu
struct CoarseDev {
  int nfree = 0;
  int npad = 0;            // nfree rounded up to the 64-wide tiles of the blocked sweep
  double* inv = nullptr;   // nfree x nfree, row-major, FP64 inverse of the coarse free-dof block
  double* X = nullptr;     // setup scratch: unit columns, their images, the dense matrix
  double* Y = nullptr;
  double* A = nullptr;     // npad x npad, swept in place (upper triangle)
  double* P = nullptr;     // npad x 64: the current pivot-column panel
  double* U = nullptr;     // npad x 64: the panel times the inverse of its diagonal block
  double* S = nullptr;     // 64 x 64: that inverse
};
int coarse_alloc(const struct LevelDev& L, CoarseDev* C);
// df64: the sweep in double-float arithmetic (mixed mode), else FP64
void coarse_setup(const struct LevelDev& L, double gamma, CoarseDev* C, struct DevStatus* st, cudaStream_t s,
                  int df64);
void coarse_apply(const struct LevelDev& L, const CoarseDev& C, int prec, const void* b, void* x, cudaStream_t s);
void coarse_free(CoarseDev* C);
// merged launches over the instances of a batch (FP32; see level.h): coarse_apply of every item
struct BCoarse {
  const struct LevelDev* L;
  const CoarseDev* C;
  const void* b;
  void* x;
};
int batch_coarse_apply(const std::vector<BCoarse>& items, cudaStream_t s);
void batch_coarse_prepare();   // before the first capture of a merged coarse apply

}  // namespace als

namespace als {
// per-cell mass blocks: W^-1 = M_K(1/mu)^-1 into winv64/winv32 (if non-NULL) and the
// Schur blocks S (if non-NULL) of variant 0 (P1) or 1 (P2), Eq. (P1P2)
void schur_setup(const struct Geom& g, double gamma, const double* mu, double* S, struct DevStatus* st, cudaStream_t s,
                 int variant = 0, double* winv64 = nullptr, float* winv32 = nullptr);
void bnd_mask(const struct Geom& g, const double* x, double* y, int keep_boundary, cudaStream_t s);
void winv_scale(const struct Geom& g, double gamma, const double* r2, double* out, cudaStream_t s,
                const double* winv = nullptr, int npr = 0);
}  // namespace als
