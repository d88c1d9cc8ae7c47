// C ABI of the AL-multigrid Stokes library: context, multigrid hierarchy,
// V-cycle (captured once per precision as a CUDA graph), block-LDU
// preconditioner and FGMRES.  Every arithmetic step runs in the kernels of
// operator.cu, patches.cu, transfer.cu, coarse.cu and krylov.cu; the host only
// sequences launches and reads one residual scalar per FGMRES iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/alstokes.h"
#include "cell.cuh"
#include "krylov.h"
#include "level.h"

using namespace als;

namespace {

struct MGWork {
  int prec = 0;
  size_t es = 8;
  std::vector<void*> b, x, t, t2, t3, scratch, V, Z;
  std::vector<double*> small;  // per level: H, cs, sn, g, y, res, beta, nrm2
  double* partial = nullptr;
  cudaGraph_t graph_tmpl = nullptr;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  // while kernels are timed: the same cycle with event-record nodes, replayed for one
  // cycle in every kProfEvery (the others replay the plain graph)
  cudaGraph_t graph_prof_tmpl = nullptr;
  cudaGraphExec_t graph_prof = nullptr;
  long long replays = 0;
};

// Live timing of finest-level kernels inside the V-cycle: kind 0 = the star-patch
// kernel (K4), kind 1 = the operator-apply cell kernel (K1, without its gather).
// The captured graph holds event-record nodes around each such launch; before
// every replay they are re-pointed at fresh events from a pool, so every launch of
// the timed region is measured with CUDA events on the stream it runs on.
struct ProfPair {
  size_t a, b;
  int kind;
};
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> slots;           // events recorded at capture time (2 per launch)
  std::vector<int> slot_kind;               // kind of each captured pair, capture order
  std::vector<cudaGraphNode_t> nodes32, nodes64;
  std::vector<int> kinds32, kinds64;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<ProfPair> pairs;
  double acc_ms[2] = {0.0, 0.0};
  long long acc_n[2] = {0, 0};
  cudaEvent_t spare0 = nullptr, spare1 = nullptr;
};

// per-level GMRES state array (GmresLayout offsets): elements of the cycle's precision in the
// fused smoother, doubles in the per-operation one
struct SmallLayout : GmresLayout {
  explicit SmallLayout(int steps) : GmresLayout(steps) {}
  GmresDev dev(double* base) const { return GmresDev{base, s}; }
};

}  // namespace

struct als_ctx {
  cudaStream_t stream = nullptr;       // internal, non-blocking
  cudaStream_t user_stream = nullptr;  // caller's stream: work is ordered after it
  cudaEvent_t order_ev = nullptr;
  int dim = 0, L = 0;
  int k = 2;             // polynomial order of the velocity (2, or 3: [Q3]^2 x P2disc)
  int npr = 0;           // pressure unknowns per cell
  int nq = 0;            // Gauss points per cell
  double gamma = 0.0;
  als_options opt{};
  std::vector<LevelDev> lev;
  CoarseDev coarse{};
  DevStatus* st = nullptr;
  double* schur = nullptr;
  MGWork w64, w32;
  // outer solve buffers (FP64), allocated on first solve
  int maxit_alloc = 0;
  long long nu = 0, np = 0, n = 0;
  double *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
  double *res = nullptr, *beta = nullptr, *h2 = nullptr, *nrm2 = nullptr, *partial = nullptr;
  double *f_dev = nullptr, *ubc_dev = nullptr, *r2_dev = nullptr, *uD = nullptr, *tu = nullptr, *tu2 = nullptr;
  double *tp = nullptr, *tp2 = nullptr, *xsol = nullptr;
  float* tp32 = nullptr;       // pressure-space vector of the FP32 B and B^T applies (mixed mode)
  double* host_res = nullptr;  // pinned
  std::vector<void*> allocs;
  std::string err;
  bool use_graph = true;
  Prof prof;
  const double* const* src_qp = nullptr;   // only valid during a setup call
  // state of the solve in progress (als_solve runs it to the end; a batch interleaves several)
  struct SolveRun {
    int k = 0, its = 0;
    double beta = 0.0, resid = 0.0;
    bool converged = false, done = false;
    als_status status = ALS_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* u = nullptr;
    double* p = nullptr;
    std::vector<double> hist;   // |b|, then the FGMRES residual estimate after each iteration
  } run;
  unsigned long long* minbits = nullptr;   // device scratch of the smallest-viscosity check
  // Newton's method (als_newton_solve): iterate, step, trial point, residual, load vector,
  // viscosity at the finest points, and the linearised coefficients of every level
  struct NewtonBuf {
    bool ready = false;
    double *u = nullptr, *p = nullptr, *du = nullptr, *dp = nullptr, *ut = nullptr, *pt = nullptr;
    double *Ru = nullptr, *Rp = nullptr, *F = nullptr, *mu = nullptr;
    std::vector<double*> C, mul;
    std::vector<double> hist;
    std::vector<int> lin;
  } nw;
};

namespace {

als_status fail(als_ctx* c, als_status code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

als_status cuda_check(als_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, ALS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return ALS_OK;
}

template <typename T>
als_status dalloc(als_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&v, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, ALS_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(v);
  *p = (T*)v;
  return ALS_OK;
}

#define ALS_TRY(expr)                 \
  do {                                \
    als_status _s = (expr);           \
    if (_s != ALS_OK) return _s;      \
  } while (0)

Geom make_geom(int dim, const int n[3], int order = 2) {
  Geom g{};
  g.dim = dim;
  for (int k = 0; k < 3; ++k) {
    const bool act = k < dim;
    g.n[k] = act ? n[k] : 1;
    g.nn[k] = act ? order * n[k] + 1 : 1;
    g.nv[k] = act ? n[k] + 1 : 1;
    g.h[k] = act ? 1.0 / n[k] : 0.0;
  }
  g.N = (long long)g.nn[0] * g.nn[1] * g.nn[2];
  g.ncells = (long long)g.n[0] * g.n[1] * g.n[2];
  g.nverts = (long long)g.nv[0] * g.nv[1] * g.nv[2];
  return g;
}

als_status check_status(als_ctx* c, const char* stage) {
  DevStatus h{};
  if (cudaMemcpyAsync(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_check(c, stage);
  if (h.code != 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: device reported status %d at index %lld", stage, h.code, h.where);
    cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream);
    return fail(c, (als_status)h.code, buf);
  }
  return ALS_OK;
}

als_status alloc_work(als_ctx* c, MGWork& w, int prec) {
  w.prec = prec;
  w.es = prec == PREC_F64 ? 8 : 4;
  const int s = std::max(1, c->opt.sweeps);
  SmallLayout sl(s);
  const int L = c->L;
  w.b.assign(L, nullptr); w.x.assign(L, nullptr); w.t.assign(L, nullptr); w.t2.assign(L, nullptr);
  w.t3.assign(L, nullptr); w.scratch.assign(L, nullptr); w.V.assign(L, nullptr); w.Z.assign(L, nullptr);
  w.small.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const size_t len = (size_t)(c->lev[l].g.N * c->dim);
    char* p = nullptr;
    ALS_TRY(dalloc(c, &p, len * w.es * 5));
    w.b[l] = p; w.x[l] = p + len * w.es; w.t[l] = p + 2 * len * w.es;
    w.t2[l] = p + 3 * len * w.es; w.t3[l] = p + 4 * len * w.es;
    if (l > 0) {
      char* q = nullptr;
      ALS_TRY(dalloc(c, &q, patch_scratch_bytes(c->lev[l], prec)));
      w.scratch[l] = q;
      ALS_TRY(dalloc(c, &q, len * w.es * (2 * s + 1)));
      w.V[l] = q;
      w.Z[l] = q + len * w.es * (s + 1);
      ALS_TRY(dalloc(c, &w.small[l], sl.total));
    }
  }
  const size_t npart = std::max(multidot_partial_doubles(std::max(s + 1, 8)),
                                 gmres_partial_doubles(c->lev[c->L - 1].g.N * c->dim));
  ALS_TRY(dalloc(c, &w.partial, npart));
  cudaMemsetAsync(w.partial, 0, sizeof(double) * npart, c->stream);
  return ALS_OK;
}

void free_graphs(als_ctx* c) {
  for (MGWork* w : {&c->w64, &c->w32}) {
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->graph_tmpl) cudaGraphDestroy(w->graph_tmpl);
    if (w->graph_prof) cudaGraphExecDestroy(w->graph_prof);
    if (w->graph_prof_tmpl) cudaGraphDestroy(w->graph_prof_tmpl);
    w->graph = nullptr;
    w->graph_tmpl = nullptr;
    w->graph_prof = nullptr;
    w->graph_prof_tmpl = nullptr;
    w->replays = 0;
  }
  c->prof.nodes32.clear();
  c->prof.nodes64.clear();
}

static thread_local bool t_capturing = false;
static thread_local bool t_capture_events = false;   // the graph being captured gets event-record nodes
cudaEvent_t prof_take(als_ctx* c);

// events for the k-th finest-level patch launch of the V-cycle being issued:
// placeholders while a graph is captured, pool events otherwise
void prof_events(als_ctx* c, int& counter, cudaEvent_t& e0, cudaEvent_t& e1, int kind = 0) {
  e0 = e1 = nullptr;
  if (!c->prof.on || (t_capturing && !t_capture_events)) return;
  if (!t_capturing) {
    e0 = prof_take(c);
    e1 = prof_take(c);
    if (e0 && e1) c->prof.pairs.push_back({c->prof.next - 2, c->prof.next - 1, kind});
    else e0 = e1 = nullptr;
    return;
  }
  const size_t need = 2 * (size_t)(counter + 1);
  while (c->prof.slots.size() < need) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->prof.slots.push_back(e);
  }
  e0 = c->prof.slots[2 * counter];
  e1 = c->prof.slots[2 * counter + 1];
  if (c->prof.slot_kind.size() < (size_t)counter + 1) c->prof.slot_kind.resize(counter + 1);
  c->prof.slot_kind[counter] = kind;
  ++counter;
}

// --------------------------------------------------------------------------
// smoothing, transfers, V-cycle (all stream-ordered, no host synchronisation)
// --------------------------------------------------------------------------
inline char* vptr(void* base, size_t es, long long off) { return (char*)base + es * off; }

static thread_local int t_prof_counter = 0;

// GMRES(s) smoothing with the fused kernels: the basis is stored unnormalised
// (column i = hn[i] v_i), the dots ride on the operator's gather, the
// Gram-Schmidt update carries the Givens step, and the final update also forms
// the residual b - A x from the Arnoldi relation when `t` is given.
bool fused_gmres(const als_ctx* c) {
  return c->opt.smoother == ALS_SMOOTH_GMRES && std::max(1, c->opt.sweeps) <= KMAXB;
}

// FP32 3D cycles form Z_j inside the operator's cell kernel from the patch outputs
// (one launch less per Arnoldi step); ALS_FUSE_GATHER=0 keeps the separate gather
bool fuse_patch_gather(const als_ctx* c, int prec) {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("ALS_FUSE_GATHER");
    v = (e && e[0] == '0') ? 0 : 1;
  }
  return v == 1 && prec == PREC_F32 && c->dim == 3 && c->k == 2;
}

void smooth_fused(als_ctx* c, MGWork& w, int l, bool x_is_zero, void* t) {
  const LevelDev& Lv = c->lev[l];
  const int prec = w.prec;
  const long long len = Lv.g.N * c->dim;
  const cudaStream_t s = c->stream;
  const int steps = std::max(1, c->opt.sweeps);
  SmallLayout sl(steps);
  double* sm = w.small[l];
  const GmresDev st = sl.dev(sm);
  void* V0 = w.V[l];
  if (x_is_zero) {
    gm_start(prec, len, w.b[l], V0, w.partial, st, s);                   // V0 = b
  } else {
    ApplyEpi e{w.b[l], -1.0, 0, nullptr, 0, nullptr, 1, st, w.partial};
    op_apply_epi(Lv, prec, c->gamma, w.x[l], V0, e, s);                  // V0 = b - A x
  }
  for (int j = 0; j < steps; ++j) {
    void* Vj = vptr(w.V[l], w.es, (long long)j * len);
    void* Vn = vptr(w.V[l], w.es, (long long)(j + 1) * len);
    void* Zj = vptr(w.Z[l], w.es, (long long)j * len);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (l == c->L - 1) prof_events(c, t_prof_counter, e0, e1);
    ApplyEpi e{nullptr, 1.0, j + 1, w.V[l], len, vptr(sm, w.es, sl.H + (long long)j * sl.ldh), 0, st, w.partial};
    if (fuse_patch_gather(c, prec)) {
      // patch products only; the cell kernel sums them per node into Z_j (= D^-1 v_j / h_j)
      patch_products(Lv, Vj, w.scratch[l], s, e0, e1);
      e.pout = w.scratch[l];
      e.pden = vptr(sm, w.es, sl.hn + j);
    } else {
      patch_smooth(Lv, prec, Vj, Zj, w.scratch[l], s, e0, e1, vptr(sm, w.es, sl.hn + j));  // Z_j = D^-1 v_j
    }
    cudaEvent_t a0 = nullptr, a1 = nullptr;
    if (l == c->L - 1) prof_events(c, t_prof_counter, a0, a1, 1);
    op_apply_epi(Lv, prec, c->gamma, Zj, Vn, e, s, a0, a1);            // A Z_j, H[0..j][j]
    gm_orth(prec, len, j, w.V[l], len, w.partial, st, s);                 // V_{j+1}, Givens step j
  }
  gm_update(prec, len, steps, w.Z[l], w.V[l], len, st, w.x[l], x_is_zero ? 1 : 0, t, s);
}

void smooth(als_ctx* c, MGWork& w, int l, bool x_is_zero = false) {
  const LevelDev& Lv = c->lev[l];
  const int prec = w.prec;
  const long long len = Lv.g.N * c->dim;
  const cudaStream_t s = c->stream;
  const int steps = std::max(1, c->opt.sweeps);
  if (c->opt.smoother == ALS_SMOOTH_RICHARDSON) {
    for (int it = 0; it < steps; ++it) {
      op_apply(Lv, prec, OP_VISC | OP_AL, c->gamma, w.x[l], w.t[l], nullptr, nullptr, s);
      vec_axpby(prec, len, 1.0, w.b[l], -1.0, w.t[l], s);                 // t = b - A x
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (l == c->L - 1) prof_events(c, t_prof_counter, e0, e1);
      patch_smooth(Lv, prec, w.t[l], w.t2[l], w.scratch[l], s, e0, e1);  // t2 = D^-1 t
      vec_axpby(prec, len, c->opt.tau, w.t2[l], 1.0, w.x[l], s);         // x += tau t2
    }
    return;
  }
  // s steps of GMRES right-preconditioned by D^-1 (classical Gram-Schmidt)
  SmallLayout sl(steps);
  double* sm = w.small[l];
  void* V0 = w.V[l];
  if (x_is_zero) {
    vec_axpby(prec, len, 1.0, w.b[l], 0.0, V0, s);                       // V0 = b (x = 0)
  } else {
    op_apply(Lv, prec, OP_VISC | OP_AL, c->gamma, w.x[l], V0, nullptr, nullptr, s);
    vec_axpby(prec, len, 1.0, w.b[l], -1.0, V0, s);                      // V0 = b - A x
  }
  vec_multidot(prec, len, 1, V0, len, V0, sm + sl.nrm2, w.partial, s);
  dev_init_g(steps + 1, sm + sl.nrm2, sm + sl.g, sm + sl.beta, s);
  vec_scale_dev(prec, len, nullptr, sm + sl.beta, V0, V0, s);
  for (int j = 0; j < steps; ++j) {
    void* Vj = vptr(w.V[l], w.es, (long long)j * len);
    void* Vn = vptr(w.V[l], w.es, (long long)(j + 1) * len);
    void* Zj = vptr(w.Z[l], w.es, (long long)j * len);
    double* hcol = sm + sl.H + (size_t)j * sl.ldh;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (l == c->L - 1) prof_events(c, t_prof_counter, e0, e1);
    patch_smooth(Lv, prec, Vj, Zj, w.scratch[l], s, e0, e1);
    op_apply(Lv, prec, OP_VISC | OP_AL, c->gamma, Zj, Vn, nullptr, nullptr, s);
    vec_multidot(prec, len, j + 1, w.V[l], len, Vn, hcol, w.partial, s);
    vec_multiaxpy_norm(prec, len, j + 1, w.V[l], len, hcol, -1.0, Vn, w.partial, sm + sl.nrm2, s);
    vec_scale_dev(prec, len, nullptr, sm + sl.nrm2, Vn, Vn, s, 1);
    dev_hess_givens(j, sm + sl.H, sl.ldh, nullptr, sm + sl.nrm2, sm + sl.cs, sm + sl.sn, sm + sl.g, sm + sl.res, s);
  }
  dev_backsolve(steps, sm + sl.H, sl.ldh, sm + sl.g, sm + sl.y, s);
  vec_multiaxpy(prec, len, steps, w.Z[l], len, sm + sl.y, w.x[l], s, 1.0);
}

// rc = P~^T rf : restrict the fine residual in w.t[l] into w.b[l-1]
void restrict_level(als_ctx* c, MGWork& w, int l, const void* rf, void* rc) {
  const LevelDev& F = c->lev[l];
  const LevelDev& C = c->lev[l - 1];
  const cudaStream_t s = c->stream;
  if (c->opt.transfer == ALS_TRANSFER_ROBUST) {
    // t2 = sum_K E_K A_K^-1 E_K^T rf ; t3 = G t2 ; rc = P_H^T (rf - t3)
    patch_interior_solve(F, w.prec, rf, w.t2[l], 0, s);
    op_apply(F, w.prec, OP_AL, c->gamma, w.t2[l], w.t3[l], nullptr, nullptr, s);
    restrict_std(C, F, w.prec, rf, rc, s, w.t3[l]);                        // P_H^T (rf - t3)
  } else {
    restrict_std(C, F, w.prec, rf, rc, s);
  }
}

// x += P~ xc with t as scratch for P_H xc; x == NULL: t = P~ xc
void prolong_level(als_ctx* c, MGWork& w, int l, const void* xc, void* t, void* x) {
  const LevelDev& F = c->lev[l];
  const LevelDev& C = c->lev[l - 1];
  const cudaStream_t s = c->stream;
  prolong_std(C, F, w.prec, xc, t, s, x);                                     // t = P_H xc, x += t
  if (c->opt.transfer == ALS_TRANSFER_ROBUST) {
    op_apply(F, w.prec, OP_AL, c->gamma, t, w.t3[l], nullptr, nullptr, s);    // t3 = G P_H xc
    patch_interior_solve(F, w.prec, w.t3[l], x ? x : t, 1, s);                // -= sum_K E A^-1 E^T t3
  }
}

// One multigrid cycle on level l for A_l x_l = b_l.  zero_guess: x_l starts at 0
// (else from its current value).  fcycle: the coarse correction is an F-cycle on
// level l-1 from zero followed by a V-cycle on level l-1 from that result (one
// exact solve when l-1 is the coarsest level); otherwise a V-cycle from zero.
void cycle_level(als_ctx* c, MGWork& w, int l, bool fcycle, bool zero_guess) {
  const cudaStream_t s = c->stream;
  if (l == 0) {
    coarse_apply(c->lev[0], c->coarse, w.prec, w.b[0], w.x[0], s);
    return;
  }
  const LevelDev& Lv = c->lev[l];
  const long long len = Lv.g.N * c->dim;
  if (fused_gmres(c) && w.prec == PREC_F32) {
    smooth_fused(c, w, l, zero_guess, w.t[l]);                           // x, and t = b - A x
  } else if (fused_gmres(c)) {
    // FP64: the residual is formed explicitly, as the method states it, not from the
    // Arnoldi relation; at extreme contrast (gamma / mu_min ~ 1e8) the recurrence drifts
    // from b - A x by far more than the rounding of b - A x itself
    smooth_fused(c, w, l, zero_guess, nullptr);
    op_apply(Lv, w.prec, OP_VISC | OP_AL, c->gamma, w.x[l], w.t[l], nullptr, nullptr, s);
    vec_axpby(w.prec, len, 1.0, w.b[l], -1.0, w.t[l], s);                // t = b - A x
  } else {
    if (zero_guess) vec_zero(w.prec, len, w.x[l], s);
    smooth(c, w, l, zero_guess && c->opt.smoother == ALS_SMOOTH_GMRES);
    op_apply(Lv, w.prec, OP_VISC | OP_AL, c->gamma, w.x[l], w.t[l], nullptr, nullptr, s);
    vec_axpby(w.prec, len, 1.0, w.b[l], -1.0, w.t[l], s);                // t = b - A x
  }
  restrict_level(c, w, l, w.t[l], w.b[l - 1]);
  cycle_level(c, w, l - 1, fcycle, true);
  if (fcycle && l - 1 > 0) cycle_level(c, w, l - 1, false, false);
  prolong_level(c, w, l, w.x[l - 1], w.t[l], w.x[l]);                  // x += P~ e_c
  if (fused_gmres(c)) smooth_fused(c, w, l, false, nullptr);
  else smooth(c, w, l);
}

cudaEvent_t prof_take(als_ctx* c) {
  Prof& p = c->prof;
  if (p.next < p.pool.size()) return p.pool[p.next++];
  return nullptr;
}

// FP32: pick the patch-kernel variant of every smoothed level (once, before capture)
void tune_patches(als_ctx* c, MGWork& w) {
  if (w.prec != PREC_F32) return;
  for (int l = 1; l < c->L; ++l) {
    LevelDev& Lv = c->lev[l];
    if (Lv.patch_kernel >= 0) continue;
    const long long len = Lv.g.N * c->dim;
    vec_zero(PREC_F32, len, w.V[l], c->stream);
    patch_autotune(Lv, w.V[l], w.scratch[l], c->stream, Lv.tune_ms);
  }
}

// Timing of the finest-level kernels samples one cycle in every kProfEvery: the
// event-record nodes split the programmatic-launch chain and every replay of the
// timed graph re-points them, so timing every cycle would slow the cycles it times.
constexpr long long kProfEvery = 8;

// capture one cycle of this precision (with_events: with the event-record nodes of
// the timed kernels) and instantiate it
static als_status capture_cycle(als_ctx* c, MGWork& w, bool with_events, cudaGraph_t* tmpl, cudaGraphExec_t* exec) {
  t_prof_counter = 0;
  const long long c0 = launch_count();
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return cuda_check(c, "begin capture");
  t_capturing = true;
  t_capture_events = with_events;
  cycle_level(c, w, c->L - 1, c->opt.cycle == ALS_CYCLE_F, true);
  t_capturing = false;
  t_capture_events = false;
  if (cudaStreamEndCapture(c->stream, tmpl) != cudaSuccess) return cuda_check(c, "end capture");
  w.graph_kernels = launch_count() - c0;
  count_launch(-w.graph_kernels);
  if (cudaGraphInstantiate(exec, *tmpl, 0) != cudaSuccess) return cuda_check(c, "graph instantiate");
  return ALS_OK;
}

// capture the cycle of this precision as a graph (once); nothing is launched
als_status ensure_graph(als_ctx* c, MGWork& w) {
  Prof& pf = c->prof;
  if (!w.graph) tune_patches(c, w);
  std::vector<cudaGraphNode_t>& nodes = w.prec == PREC_F64 ? pf.nodes64 : pf.nodes32;
  std::vector<int>& kinds = w.prec == PREC_F64 ? pf.kinds64 : pf.kinds32;
  if (!w.graph) {
    ALS_TRY(capture_cycle(c, w, false, &w.graph_tmpl, &w.graph));
    nodes.clear();
    w.replays = 0;
  }
  if (pf.on && !w.graph_prof) {
    ALS_TRY(capture_cycle(c, w, true, &w.graph_prof_tmpl, &w.graph_prof));
    // map every event-record node to its slot (capture order is the slot order)
    const int nslots = 2 * t_prof_counter;
    nodes.assign(nslots, nullptr);
    kinds.assign(pf.slot_kind.begin(), pf.slot_kind.begin() + t_prof_counter);
    size_t nn = 0;
    cudaGraphGetNodes(w.graph_prof_tmpl, nullptr, &nn);
    std::vector<cudaGraphNode_t> all(nn);
    cudaGraphGetNodes(w.graph_prof_tmpl, all.data(), &nn);
    for (cudaGraphNode_t nd : all) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev;
      cudaGraphEventRecordNodeGetEvent(nd, &ev);
      for (int i = 0; i < nslots; ++i)
        if (pf.slots[i] == ev) nodes[i] = nd;
    }
  }
  return ALS_OK;
}

// one cycle on the finest level: w.b[L-1] -> w.x[L-1]
als_status run_vcycle(als_ctx* c, MGWork& w) {
  Prof& pf = c->prof;
  if (!c->use_graph) {
    tune_patches(c, w);
    cycle_level(c, w, c->L - 1, c->opt.cycle == ALS_CYCLE_F, true);
    return cuda_check(c, "vcycle");
  }
  ALS_TRY(ensure_graph(c, w));
  std::vector<cudaGraphNode_t>& nodes = w.prec == PREC_F64 ? pf.nodes64 : pf.nodes32;
  std::vector<int>& kinds = w.prec == PREC_F64 ? pf.kinds64 : pf.kinds32;
  cudaGraphExec_t exec = w.graph;
  if (pf.on && w.graph_prof && !nodes.empty() && w.replays % kProfEvery == 0) {
    exec = w.graph_prof;
    for (size_t i = 0; i + 1 < nodes.size(); i += 2) {
      cudaEvent_t a = prof_take(c), b = prof_take(c);
      if (!a || !b) { a = pf.spare0; b = pf.spare1; }
      else pf.pairs.push_back({pf.next - 2, pf.next - 1, kinds[i / 2]});
      if (nodes[i]) cudaGraphExecEventRecordNodeSetEvent(exec, nodes[i], a);
      if (nodes[i + 1]) cudaGraphExecEventRecordNodeSetEvent(exec, nodes[i + 1], b);
    }
  }
  ++w.replays;
  if (cudaGraphLaunch(exec, c->stream) != cudaSuccess) return cuda_check(c, "graph launch");
  count_launch(w.graph_kernels);
  return ALS_OK;
}

MGWork& work_for(als_ctx* c, int prec) { return prec == PREC_F64 ? c->w64 : c->w32; }

// --------------------------------------------------------------------------
// outer solve
// --------------------------------------------------------------------------
als_status alloc_solve(als_ctx* c, int maxit) {
  if (c->maxit_alloc >= maxit) return ALS_OK;
  if (c->maxit_alloc > 0) return fail(c, ALS_EINVAL, "maxit larger than the first solve's is not supported");
  const LevelDev& F = c->lev[c->L - 1];
  c->nu = F.g.N * c->dim;
  c->np = F.g.ncells * c->npr;
  c->n = c->nu + c->np;
  const int ldh = maxit + 1;
  ALS_TRY(dalloc(c, &c->V, (size_t)(maxit + 1) * c->n));
  ALS_TRY(dalloc(c, &c->Z, (size_t)maxit * c->n));
  ALS_TRY(dalloc(c, &c->H, (size_t)ldh * maxit));
  ALS_TRY(dalloc(c, &c->cs, maxit));
  ALS_TRY(dalloc(c, &c->sn, maxit));
  ALS_TRY(dalloc(c, &c->g, maxit + 1));
  ALS_TRY(dalloc(c, &c->y, maxit));
  ALS_TRY(dalloc(c, &c->res, 1));
  ALS_TRY(dalloc(c, &c->beta, 1));
  ALS_TRY(dalloc(c, &c->h2, maxit + 1));
  ALS_TRY(dalloc(c, &c->nrm2, 1));
  ALS_TRY(dalloc(c, &c->partial, multidot_partial_doubles(maxit + 1)));
  cudaMemsetAsync(c->partial, 0, sizeof(double) * multidot_partial_doubles(maxit + 1), c->stream);
  ALS_TRY(dalloc(c, &c->f_dev, (size_t)F.g.ncells * c->nq * c->dim));
  ALS_TRY(dalloc(c, &c->ubc_dev, c->nu));
  ALS_TRY(dalloc(c, &c->r2_dev, c->np));
  ALS_TRY(dalloc(c, &c->uD, c->nu));
  ALS_TRY(dalloc(c, &c->tu, c->nu));
  ALS_TRY(dalloc(c, &c->tu2, c->nu));
  ALS_TRY(dalloc(c, &c->tp, c->np));
  ALS_TRY(dalloc(c, &c->tp2, c->np));
  ALS_TRY(dalloc(c, &c->tp32, c->np));
  ALS_TRY(dalloc(c, &c->xsol, c->n));
  if (!c->host_res && cudaMallocHost(&c->host_res, 2 * sizeof(double)) != cudaSuccess)
    return fail(c, ALS_ENOMEM, "pinned host allocation failed");
  c->maxit_alloc = maxit;
  return ALS_OK;
}

// z1 = A^-1 f through one V-cycle in the context's precision mode (FP64 in/out)
als_status apply_Ahat(als_ctx* c, const double* f, double* z1) {
  const int prec = c->opt.mode == ALS_MODE_MIXED ? PREC_F32 : PREC_F64;
  MGWork& w = work_for(c, prec);
  const int l = c->L - 1;
  vec_cast(c->nu, f, PREC_F64, w.b[l], prec, c->stream);
  ALS_TRY(run_vcycle(c, w));
  vec_cast(c->nu, w.x[l], prec, z1, PREC_F64, c->stream);
  return ALS_OK;
}

// Eq. (precond): z = P v, v = (f, g), z = (x1, z2)
als_status precondition(als_ctx* c, const double* v, double* z) {
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  const double* f = v;
  const double* gp = v + c->nu;
  double* x1 = z;
  double* z2 = z + c->nu;
  if (c->opt.fact != ALS_FACT_FULL) {
    // the factorisation types with one (1,1) application (oracle: StokesSolver.precondition)
    if (c->opt.fact == ALS_FACT_UPPER) {                        // [[A, B^T], [0, -S]]^-1
      schur_apply(F.g.ncells, c->npr, c->schur, gp, z2, s);                      // z2 = -S^-1 g
      op_apply(F, PREC_F64, OP_BT, c->gamma, nullptr, c->tu2, z2, nullptr, s);         // tu2 = B^T z2
      vec_axpby(PREC_F64, c->nu, 1.0, f, -1.0, c->tu2, s);                             // tu2 = f - tu2
      ALS_TRY(apply_Ahat(c, c->tu2, x1));                                              // x1 = A^-1 tu2
    } else {
      ALS_TRY(apply_Ahat(c, f, x1));                                                   // x1 = A^-1 f
      if (c->opt.fact == ALS_FACT_LOWER) {                      // [[A, 0], [B, -S]]^-1
        op_apply(F, PREC_F64, OP_B, c->gamma, x1, nullptr, nullptr, c->tp, s);        // tp = B x1
        vec_axpby(PREC_F64, c->np, 1.0, gp, -1.0, c->tp, s);                           // tp = g - B x1
        schur_apply(F.g.ncells, c->npr, c->schur, c->tp, z2, s);                   // z2 = -S^-1 tp
      } else {                                                  // diag(A^-1, -S^-1)
        schur_apply(F.g.ncells, c->npr, c->schur, gp, z2, s);                      // z2 = -S^-1 g
      }
    }
    project_constant(F.g.ncells, c->npr, z2, c->partial, s);
    return ALS_OK;
  }
  if (c->opt.mode == ALS_MODE_MIXED) {
    // The off-diagonal blocks run in the precision of the cycle: B reads the FP32
    // cycle output directly and B^T writes the right-hand side of the second cycle,
    // while g - B z1, the Schur blocks and the final combination stay in FP64.
    MGWork& w = work_for(c, PREC_F32);
    const int l = c->L - 1;
    vec_cast(c->nu, f, PREC_F64, w.b[l], PREC_F32, s);
    ALS_TRY(run_vcycle(c, w));                                                       // z1 = A^-1 f (FP32)
    vec_cast(c->nu, w.x[l], PREC_F32, c->tu, PREC_F64, s);
    op_apply(F, PREC_F32, OP_B, c->gamma, w.x[l], nullptr, nullptr, c->tp32, s);     // B z1 (FP32)
    vec_cast(c->np, c->tp32, PREC_F32, c->tp, PREC_F64, s);
    vec_axpby(PREC_F64, c->np, 1.0, gp, -1.0, c->tp, s);                             // tp = g - B z1
    schur_apply(F.g.ncells, c->npr, c->schur, c->tp, z2, s);                     // z2 = -S^-1 tp
    vec_cast(c->np, z2, PREC_F64, c->tp32, PREC_F32, s);
    op_apply(F, PREC_F32, OP_BT, c->gamma, nullptr, w.b[l], c->tp32, nullptr, s);    // B^T z2 (FP32)
    ALS_TRY(run_vcycle(c, w));                                                       // A^-1 B^T z2 (FP32)
    vec_cast(c->nu, w.x[l], PREC_F32, x1, PREC_F64, s);
    vec_axpby(PREC_F64, c->nu, 1.0, c->tu, -1.0, x1, s);                             // x1 = z1 - x1
    project_constant(F.g.ncells, c->npr, z2, c->partial, s);
    return ALS_OK;
  }
  ALS_TRY(apply_Ahat(c, f, c->tu));                                                  // z1 = A^-1 f
  op_apply(F, PREC_F64, OP_B, c->gamma, c->tu, nullptr, nullptr, c->tp, s);          // tp = B z1
  vec_axpby(PREC_F64, c->np, 1.0, gp, -1.0, c->tp, s);                               // tp = g - B z1
  schur_apply(F.g.ncells, c->npr, c->schur, c->tp, z2, s);                       // z2 = -S^-1 tp
  op_apply(F, PREC_F64, OP_BT, c->gamma, nullptr, c->tu2, z2, nullptr, s);           // tu2 = B^T z2
  ALS_TRY(apply_Ahat(c, c->tu2, x1));                                                // x1 = A^-1 B^T z2
  vec_axpby(PREC_F64, c->nu, 1.0, c->tu, -1.0, x1, s);                               // x1 = z1 - x1
  project_constant(F.g.ncells, c->npr, z2, c->partial, s);
  return ALS_OK;
}

void matvec(als_ctx* c, const double* x, double* y) {
  const LevelDev& F = c->lev[c->L - 1];
  op_apply(F, PREC_F64, OP_VISC | OP_AL | OP_BT | OP_B, c->gamma, x, y, x + c->nu, y + c->nu, c->stream);
}

// No C++ exception crosses the C ABI: every entry point that returns a status is a
// function-try-block whose handler maps the exception in flight (host containers and
// strings can throw std::bad_alloc) to a status.  A failure there leaves whatever the
// call had changed, like any other mid-call failure.
als_status caught_exception() noexcept {
  try {
    throw;
  } catch (const std::bad_alloc&) {
    return ALS_ENOMEM;
  } catch (...) {
    return ALS_EINVAL;
  }
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

void als_default_options(als_options* opt) {
  if (!opt) return;
  opt->smoother = ALS_SMOOTH_GMRES;
  opt->sweeps = 5;
  opt->tau = 0.0;
  opt->transfer = ALS_TRANSFER_ROBUST;
  opt->schur = ALS_SCHUR_P1;
  opt->mode = ALS_MODE_FP64;
  opt->rtol = 1e-8;
  opt->maxit = 300;
  opt->cycle = ALS_CYCLE_V;
  opt->fact = ALS_FACT_FULL;
  opt->setup = ALS_SETUP_AUTO;
  opt->order = 2;
  opt->store = ALS_STORE_FP32;
}

// message of the calling thread's last failed als_create (the context is gone by then)
static thread_local std::string t_create_err;

const char* als_last_error(const als_ctx* ctx) { return ctx ? ctx->err.c_str() : t_create_err.c_str(); }

als_status als_destroy(als_ctx* ctx) try {
  if (!ctx) return ALS_EINVAL;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_graphs(ctx);
  coarse_free(&ctx->coarse);
  for (cudaEvent_t e : ctx->prof.slots) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
  if (ctx->prof.spare0) cudaEventDestroy(ctx->prof.spare0);
  if (ctx->prof.spare1) cudaEventDestroy(ctx->prof.spare1);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->host_res) cudaFreeHost(ctx->host_res);
  if (ctx->order_ev) cudaEventDestroy(ctx->order_ev);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

// Setup (Secs. 4-5) with the coefficients of every level: copies them, builds
// the vertex-star patch inverses, the coarse factorisation and the Schur blocks.
// Smallest viscosity of all levels' points (mu, or mu_eff for tensor coefficients).
// The FP32 cycle of the P1 pairing (augmentation weight W = M_p) evaluates the AL
// term gamma div u beside viscous terms of size mu_min in single precision; once
// 2^-24 gamma / mu_min exceeds 0.1 it no longer converges (measured on the 3D 32^3
// sinker problem at DR 1e6 and 1e8), so mixed mode refuses that pairing there; the
// P2 pairing (W = M_p(1/mu)) scales the AL term with mu and has no such limit.
static als_status check_mixed_range(als_ctx* c) {
  if (c->opt.mode != ALS_MODE_MIXED || c->opt.schur != ALS_SCHUR_P1 || c->gamma == 0.0) return ALS_OK;
  const int NB = c->nq;
  const unsigned long long inf_bits = 0x7ff0000000000000ull;
  cudaMemcpyAsync(c->minbits, &inf_bits, sizeof(inf_bits), cudaMemcpyHostToDevice, c->stream);
  for (int l = 0; l < c->L; ++l)
    vec_min_positive(c->lev[l].g.ncells * NB, c->lev[l].mu64, c->minbits, c->stream);
  unsigned long long bits = inf_bits;
  if (cudaMemcpyAsync(&bits, c->minbits, sizeof(bits), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_check(c, "viscosity range");
  double mu_min;
  memcpy(&mu_min, &bits, sizeof(mu_min));
  const double lim = 0.1 / std::ldexp(1.0, -24);   // gamma / mu_min above which the FP32 P1 cycle fails
  if (c->gamma / mu_min > lim) {
    char buf[320];
    snprintf(buf, sizeof(buf),
             "mixed precision with the P1 pairing needs 2^-24 gamma / mu_min <= 0.1 (gamma / mu_min = %.3g > %.3g): "
             "use ALS_SCHUR_P2 (W = M_p(1/mu)) or ALS_MODE_FP64",
             c->gamma / mu_min, lim);
    return fail(c, ALS_EINVAL, buf);
  }
  return ALS_OK;
}

static als_status run_setup(als_ctx* c, const als_coeff* coeff) {
  const int NB = c->nq;
  // FP64 or double-float arithmetic for the patch and coarse inverses
  const int df64 = c->opt.mode == ALS_MODE_MIXED && c->opt.setup != ALS_SETUP_FP64 ? 1 : 0;
  for (int l = 0; l < c->L; ++l) {
    LevelDev& Lv = c->lev[l];
    const size_t ncq = (size_t)Lv.g.ncells * NB * Lv.ncoef;
    if (!coeff->qp[l]) return fail(c, ALS_EINVAL, "missing coefficients for a level");
    if (cudaMemcpyAsync(Lv.coef64, coeff->qp[l], ncq * sizeof(double), cudaMemcpyDefault, c->stream) != cudaSuccess)
      return cuda_check(c, "copy coefficients");
    vec_cast((long long)ncq, Lv.coef64, PREC_F64, Lv.coef32, PREC_F32, c->stream);
    if (Lv.tensor) {
      if (!coeff->mu_eff[l]) return fail(c, ALS_EINVAL, "missing mu_eff for a level");
      const size_t nq = (size_t)Lv.g.ncells * NB;
      if (cudaMemcpyAsync(Lv.mu64, coeff->mu_eff[l], nq * sizeof(double), cudaMemcpyDefault, c->stream) != cudaSuccess)
        return cuda_check(c, "copy mu_eff");
    }
  }
  ALS_TRY(check_mixed_range(c));
  if (c->k == 3) {
    // order 3: per-cell W^-1 of every level (the AL term of the operator and the stars) and
    // the finest level's Schur blocks, then the stars (FP64 assembly; the 3D elimination in
    // double-float when df64, else FP64) and the coarse inverse
    const int p2 = c->opt.schur == ALS_SCHUR_P2 ? 1 : 0;
    for (int l = 0; l < c->L; ++l) {
      LevelDev& Lv = c->lev[l];
      qk_mass_setup(Lv, c->gamma, p2, p2, Lv.winv64, Lv.winv32, l == c->L - 1 ? c->schur : nullptr, c->st, c->stream);
      if (l > 0) patch_setup(Lv, c->gamma, 1, df64, c->st, c->stream);
      ALS_TRY(cuda_check(c, "order-3 setup"));
    }
    coarse_setup(c->lev[0], c->gamma, &c->coarse, c->st, c->stream, df64);
    ALS_TRY(cuda_check(c, "coarse setup"));
    return check_status(c, "setup");
  }
  for (int l = 0; l < c->L; ++l) {
    LevelDev& Lv = c->lev[l];
    if (Lv.winv64) {
      schur_setup(Lv.g, c->gamma, Lv.mu64, nullptr, c->st, c->stream, 1, Lv.winv64, Lv.winv32);
      ALS_TRY(cuda_check(c, "mass blocks"));
    }
    if (l > 0) {
      patch_setup(Lv, c->gamma, 1, df64, c->st, c->stream);
      ALS_TRY(cuda_check(c, "patch setup"));
    }
  }
  coarse_setup(c->lev[0], c->gamma, &c->coarse, c->st, c->stream, df64);
  ALS_TRY(cuda_check(c, "coarse setup"));
  const LevelDev& F = c->lev[c->L - 1];
  schur_setup(F.g, c->gamma, F.mu64, c->schur, c->st, c->stream, c->opt.schur == ALS_SCHUR_P2 ? 1 : 0);
  ALS_TRY(cuda_check(c, "schur setup"));
  return check_status(c, "setup");
}

// FP32 star storage of a smoothed level.  Levels of at least kSplitVertices vertices use
// split storage: block-packed inverses of the interior vertices, and the boundary vertices'
// compact inverses (free dofs only: 1/3, 1/9 and 1/27 of an interior star's dofs at faces,
// edges and corners in 3D) with their vertex ids and offsets, enumerated here on the host;
// the smoother streams 15-20 % fewer bytes there and applies the boundary stars in a
// small second kernel.  Smaller levels, whose cycle time is launch latency rather than
// bytes, keep every vertex's block-packed inverse (identity rows at absent nodes) and one
// kernel.
constexpr long long kSplitVertices = 32768;

static als_status alloc_star_storage(als_ctx* c, LevelDev& Lv) {
  const Geom& g = Lv.g;
  const int d = c->dim;
  if (c->k == 3) {   // order 3: an FP32 copy of every star, in wrapped rows
    Lv.split = 0;
    Lv.nbnd = 0;
    return dalloc(c, &Lv.inv32, (size_t)g.nverts * qk_star32_floats(d));
  }
  Lv.nint = 1;
  for (int k = 0; k < d; ++k) Lv.nint *= g.nv[k] - 2;
  static int forced = -2;   // ALS_SPLIT_STARS=1 / 0 forces split / full storage on every level
  if (forced == -2) {
    const char* e = getenv("ALS_SPLIT_STARS");
    forced = (e && e[0] == '1') ? 1 : ((e && e[0] == '0') ? 0 : -1);
  }
  Lv.split = forced >= 0 ? forced : (g.nverts >= kSplitVertices ? 1 : 0);
  if (!Lv.split) {
    Lv.nbnd = 0;
    return dalloc(c, &Lv.inv32, (size_t)g.nverts * Lv.pstride);
  }
  std::vector<int> bvid;
  std::vector<long long> boff;
  long long total = 0;
  for (long long v = 0; v < g.nverts; ++v) {
    const int vc[3] = {(int)(v % g.nv[0]), (int)((v / g.nv[0]) % g.nv[1]),
                       (int)(v / ((long long)g.nv[0] * g.nv[1]))};
    int m = d;
    bool bnd = false;
    for (int k = 0; k < d; ++k) {
      const bool edge = vc[k] == 0 || vc[k] == g.nv[k] - 1;
      bnd = bnd || edge;
      m *= edge ? 1 : 3;
    }
    if (!bnd) continue;
    bvid.push_back((int)v);
    boff.push_back(total);
    total += ((long long)m * (m + 1) / 2 + 3) & ~3LL;   // 16-byte aligned blocks (bulk copies)
  }
  Lv.nbnd = (long long)bvid.size();
  ALS_TRY(dalloc(c, &Lv.inv32, (size_t)Lv.nint * Lv.pstride));
  ALS_TRY(dalloc(c, &Lv.bnd32, (size_t)total));
  ALS_TRY(dalloc(c, &Lv.bvid, bvid.size()));
  ALS_TRY(dalloc(c, &Lv.boff, boff.size()));
  if (!bvid.empty() &&
      (cudaMemcpyAsync(Lv.bvid, bvid.data(), bvid.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream) !=
           cudaSuccess ||
       cudaMemcpyAsync(Lv.boff, boff.data(), boff.size() * sizeof(long long), cudaMemcpyHostToDevice, c->stream) !=
           cudaSuccess ||
       cudaStreamSynchronize(c->stream) != cudaSuccess))
    return cuda_check(c, "boundary star tables");
  return ALS_OK;
}

static als_status create_impl(als_ctx* c, const als_mesh* mesh, const als_coeff* coeff, double gamma,
                               const als_options* opt) {
  if (!mesh || !coeff || !coeff->qp) return fail(c, ALS_EINVAL, "null mesh or coefficients");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(c, ALS_EINVAL, "dim must be 2 or 3");
  if (mesh->levels < 1 || mesh->levels > 12) return fail(c, ALS_EINVAL, "levels must be in [1, 12]");
  if (!(gamma >= 0.0) || !std::isfinite(gamma)) return fail(c, ALS_EINVAL, "gamma must be finite and >= 0");
  if (coeff->kind != ALS_COEFF_SCALAR && coeff->kind != ALS_COEFF_TENSOR)
    return fail(c, ALS_EINVAL, "unknown coefficient kind");
  if (coeff->kind == ALS_COEFF_TENSOR && !coeff->mu_eff)
    return fail(c, ALS_EINVAL, "tensor coefficients need mu_eff");
  c->dim = mesh->dim;
  c->L = mesh->levels;
  c->gamma = gamma;
  if (opt) c->opt = *opt; else als_default_options(&c->opt);
  if (c->opt.sweeps < 1 || c->opt.sweeps > 64) return fail(c, ALS_EINVAL, "sweeps must be in [1, 64]");
  if (c->opt.tau <= 0.0) c->opt.tau = std::pow(2.0, -c->dim);
  if (c->opt.maxit < 1 || c->opt.maxit > 2000) return fail(c, ALS_EINVAL, "maxit must be in [1, 2000]");
  if (c->opt.schur != ALS_SCHUR_P1 && c->opt.schur != ALS_SCHUR_P2) return fail(c, ALS_EINVAL, "unknown Schur variant");
  if (c->opt.cycle != ALS_CYCLE_V && c->opt.cycle != ALS_CYCLE_F) return fail(c, ALS_EINVAL, "unknown cycle");
  if (c->opt.fact < ALS_FACT_FULL || c->opt.fact > ALS_FACT_DIAG)
    return fail(c, ALS_EINVAL, "unknown factorisation type");
  if (c->opt.smoother != ALS_SMOOTH_GMRES && c->opt.smoother != ALS_SMOOTH_RICHARDSON)
    return fail(c, ALS_EINVAL, "unknown smoother");
  if (c->opt.transfer != ALS_TRANSFER_ROBUST && c->opt.transfer != ALS_TRANSFER_STANDARD)
    return fail(c, ALS_EINVAL, "unknown transfer");
  if (c->opt.mode != ALS_MODE_FP64 && c->opt.mode != ALS_MODE_MIXED) return fail(c, ALS_EINVAL, "unknown mode");
  if (c->opt.setup != ALS_SETUP_AUTO && c->opt.setup != ALS_SETUP_FP64)
    return fail(c, ALS_EINVAL, "unknown setup arithmetic");
  if (c->opt.store != ALS_STORE_FP32 && c->opt.store != ALS_STORE_BF16)
    return fail(c, ALS_EINVAL, "unknown star storage");
  if (c->opt.store == ALS_STORE_BF16 && c->opt.order != 2 && !(c->opt.order == 3 && c->dim == 3))
    return fail(c, ALS_EINVAL, "bfloat16 star storage is built for order 2 and for order 3 in 3D");
  if (c->opt.order != 2 && c->opt.order != 3) return fail(c, ALS_EINVAL, "order must be 2 or 3");
  if (c->opt.order == 3 && coeff->kind != ALS_COEFF_SCALAR)
    return fail(c, ALS_EINVAL, "order 3 is built for scalar viscosity");
  c->k = c->opt.order;
  c->npr = c->k == 3 ? (c->dim == 2 ? 6 : 10) : c->dim + 1;   // C(k - 1 + d, d)
  c->nq = c->k == 3 ? (c->dim == 2 ? 16 : 64) : (c->dim == 2 ? 9 : 27);
  const int f = 1 << (c->L - 1);
  for (int k = 0; k < c->dim; ++k) {
    if (mesh->n[k] < 2 || mesh->n[k] % f != 0 || mesh->n[k] / f < 2)
      return fail(c, ALS_EINVAL, "n must be divisible by 2^(levels-1) with >= 2 coarse cells per direction");
  }
  {
    long long nu = c->dim;   // vector kernels index velocity entries with 32 bits
    for (int k = 0; k < c->dim; ++k) nu *= (long long)c->k * mesh->n[k] + 1;
    if (nu >= (1LL << 31)) return fail(c, ALS_EINVAL, "mesh too large: d (k n+1)^d must stay below 2^31");
    long long ne = (long long)c->dim * c->nq;   // per-cell output buffer, 32-bit offsets
    for (int k = 0; k < c->dim; ++k) ne *= mesh->n[k];
    if (ne >= (1LL << 31)) return fail(c, ALS_EINVAL, "mesh too large: d (k+1)^d n^d must stay below 2^31");
    long long np = c->dim;   // vertex-star patch outputs, 32-bit offsets
    for (int k = 0; k < c->dim; ++k) np *= (2LL * c->k - 1) * (mesh->n[k] + 1LL);
    if (np >= (1LL << 31)) return fail(c, ALS_EINVAL, "mesh too large: d (2k-1)^d (n+1)^d must stay below 2^31");
  }
  const char* ng = getenv("ALS_NO_GRAPH");
  c->use_graph = !(ng && ng[0] == '1');
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_check(c, "stream create");
  if (cudaEventCreateWithFlags(&c->order_ev, cudaEventDisableTiming) != cudaSuccess)
    return cuda_check(c, "event create");
  ALS_TRY(dalloc(c, &c->st, 1));
  cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream);
  ALS_TRY(dalloc(c, &c->minbits, 1));
  const int NB = c->nq;
  const int NC = c->dim == 2 ? 6 : 21;
  int nstar = c->dim;   // star dofs: d (2k-1)^d
  for (int k = 0; k < c->dim; ++k) nstar *= 2 * c->k - 1;
  if (c->k == 3) qk_tables();
  c->lev.resize(c->L);
  for (int l = 0; l < c->L; ++l) {
    int nl[3] = {1, 1, 1};
    for (int k = 0; k < c->dim; ++k) nl[k] = mesh->n[k] >> (c->L - 1 - l);
    LevelDev& Lv = c->lev[l];
    Lv = LevelDev{};
    Lv.g = make_geom(c->dim, nl, c->k);
    Lv.k = c->k;
    Lv.npr = c->npr;
    Lv.nq = c->nq;
    Lv.patch_kernel = -1;
    Lv.tensor = coeff->kind == ALS_COEFF_TENSOR;
    Lv.ncoef = Lv.tensor ? NC : 1;
    Lv.np = nstar;
    Lv.pstride = packed_stride(Lv.np);
    Lv.status = c->st;
    const size_t ncq = (size_t)Lv.g.ncells * NB * Lv.ncoef;
    {
      char* tab = nullptr;
      ALS_TRY(dalloc(c, &tab, setup_tab_bytes(c->dim)));
      Lv.setup_tab = tab;
    }
    ALS_TRY(dalloc(c, &Lv.coef64, ncq));
    ALS_TRY(dalloc(c, &Lv.coef32, ncq));
    if (Lv.tensor) ALS_TRY(dalloc(c, &Lv.mu64, (size_t)Lv.g.ncells * NB));
    else Lv.mu64 = Lv.coef64;
    {
      double* e = nullptr;
      ALS_TRY(dalloc(c, &e, (size_t)Lv.g.ncells * NB * c->dim));
      Lv.ebuf = e;
    }
    if (c->opt.schur == ALS_SCHUR_P2 || c->k == 3) {   // P2: W = M_p(1/mu); order 3: per-cell W^-1 always
      const size_t nb2 = (size_t)Lv.g.ncells * c->npr * c->npr;
      ALS_TRY(dalloc(c, &Lv.winv64, nb2));
      ALS_TRY(dalloc(c, &Lv.winv32, nb2));
    }
    if (l > 0) {
      ALS_TRY(dalloc(c, &Lv.inv64, (size_t)Lv.g.nverts * Lv.pstride));
      ALS_TRY(alloc_star_storage(c, Lv));
      if (c->opt.store == ALS_STORE_BF16) {   // the FP32 stars again, in bfloat16
        uint16_t* p16 = nullptr;
        const size_t per = c->k == 3 ? qk3_star32_floats() : (size_t)block_stride_bf16(Lv.np);
        ALS_TRY(dalloc(c, &p16, (size_t)(Lv.split ? Lv.nint : Lv.g.nverts) * per));
        Lv.inv16 = p16;
      }
    }
  }
  if (c->k == 3 && c->dim == 3 && c->L > 1) {   // one star-setup workspace for all levels
    const int ctas = qk3_setup_ctas(c->lev[c->L - 1].g.nverts);
    double* ws = nullptr;
    ALS_TRY(dalloc(c, &ws, qk3_setup_ws_doubles(ctas)));
    for (int l = 1; l < c->L; ++l) {
      c->lev[l].qk_ws = ws;
      c->lev[l].qk_ws_ctas = ctas;
    }
  }
  if (coarse_alloc(c->lev[0], &c->coarse) != 0) {
    cudaGetLastError();
    return fail(c, ALS_ENOMEM, "coarse setup allocation failed");
  }
  const LevelDev& F = c->lev[c->L - 1];
  ALS_TRY(dalloc(c, &c->schur, (size_t)F.g.ncells * c->npr * c->npr));
  ALS_TRY(alloc_work(c, c->w64, PREC_F64));
  ALS_TRY(alloc_work(c, c->w32, PREC_F32));
  return run_setup(c, coeff);
}

als_status als_create(const als_mesh* mesh, const als_coeff* coeff, double gamma, const als_options* opt,
                      void* stream, als_ctx** out) try {
  t_create_err.clear();
  if (!out) {
    t_create_err = "null output pointer";
    return ALS_EINVAL;
  }
  *out = nullptr;
  als_ctx* c = new als_ctx();
  c->user_stream = (cudaStream_t)stream;
  if (stream) cudaStreamSynchronize((cudaStream_t)stream);
  als_status st = create_impl(c, mesh, coeff, gamma, opt);
  if (st != ALS_OK) {
    t_create_err = c->err;   // read back with als_last_error(NULL): the context is gone
    als_destroy(c);
    return st;
  }
  *out = c;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_update_coefficients(als_ctx* c, const als_coeff* coeff) try {
  if (!c || !coeff || !coeff->qp) return c ? fail(c, ALS_EINVAL, "null coefficients") : ALS_EINVAL;
  if ((coeff->kind == ALS_COEFF_TENSOR) != (c->lev[0].tensor != 0))
    return fail(c, ALS_EINVAL, "coefficient kind differs from the one the context was created with");
  if (coeff->kind == ALS_COEFF_TENSOR && !coeff->mu_eff) return fail(c, ALS_EINVAL, "tensor coefficients need mu_eff");
  cudaEventRecord(c->order_ev, c->user_stream);
  cudaStreamWaitEvent(c->stream, c->order_ev, 0);
  return run_setup(c, coeff);
} catch (...) {
  return caught_exception();
}

als_status als_profile(als_ctx* c, int on) try {
  if (!c) return ALS_EINVAL;
  Prof& p = c->prof;
  if ((on != 0) == p.on) return ALS_OK;
  cudaStreamSynchronize(c->stream);
  free_graphs(c);  // the V-cycle graphs are recaptured with (or without) event nodes
  p.on = on != 0;
  if (p.on && p.pool.empty()) {
    p.pool.resize(16384);
    for (auto& e : p.pool)
      if (cudaEventCreate(&e) != cudaSuccess) return cuda_check(c, "profiling events");
    cudaEventCreate(&p.spare0);
    cudaEventCreate(&p.spare1);
  }
  p.next = 0;
  p.pairs.clear();
  p.acc_ms[0] = p.acc_ms[1] = 0.0;
  p.acc_n[0] = p.acc_n[1] = 0;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

// moves the recorded pairs into the per-kind accumulators
static als_status prof_drain(als_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "profile read");
  for (auto& pr : c->prof.pairs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof.pool[pr.a], c->prof.pool[pr.b]) == cudaSuccess) {
      c->prof.acc_ms[pr.kind] += ms;
      c->prof.acc_n[pr.kind] += 1;
    } else {
      cudaGetLastError();  // an unrecorded pair is skipped, not left as a sticky error
    }
  }
  c->prof.pairs.clear();
  c->prof.next = 0;
  return ALS_OK;
}

als_status als_profile_read_kernel(als_ctx* c, int kind, double* total_ms, long long* launches) try {
  if (!c || !total_ms || !launches) return c ? fail(c, ALS_EINVAL, "null output") : ALS_EINVAL;
  if (kind < 0 || kind > 1) return fail(c, ALS_EINVAL, "kind must be 0 (patch kernel) or 1 (operator apply)");
  ALS_TRY(prof_drain(c));
  *total_ms = c->prof.acc_ms[kind];
  *launches = c->prof.acc_n[kind];
  c->prof.acc_ms[kind] = 0.0;
  c->prof.acc_n[kind] = 0;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_profile_read(als_ctx* c, double* total_ms, long long* launches) try {
  return als_profile_read_kernel(c, 0, total_ms, launches);
} catch (...) {
  return caught_exception();
}

long long als_kernel_launches(void) { return launch_count(); }

static als_status check_level(als_ctx* c, int level, int prec) {
  if (!c) return ALS_EINVAL;
  if (level < 0 || level >= c->L) return fail(c, ALS_EINVAL, "level out of range");
  if (prec != PREC_F64 && prec != PREC_F32) return fail(c, ALS_EINVAL, "prec must be ALS_PREC_FP64 or ALS_PREC_FP32");
  return ALS_OK;
}

// order the context's stream after the work already queued on the caller's stream
static void begin(als_ctx* c) {
  cudaEventRecord(c->order_ev, c->user_stream);
  cudaStreamWaitEvent(c->stream, c->order_ev, 0);
}

static als_status finish(als_ctx* c, const char* what) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, what);
  ALS_TRY(cuda_check(c, what));
  return check_status(c, what);
}

als_status als_apply_agamma(als_ctx* c, int level, int prec, const void* x, void* y) try {
  ALS_TRY(check_level(c, level, prec));
  if (!x || !y) return fail(c, ALS_EINVAL, "null vector");
  begin(c);
  op_apply(c->lev[level], prec, OP_VISC | OP_AL, c->gamma, x, y, nullptr, nullptr, c->stream);
  return finish(c, "apply_agamma");
} catch (...) {
  return caught_exception();
}

als_status als_vcycle(als_ctx* c, int prec, const void* b, void* x) try {
  ALS_TRY(check_level(c, c ? c->L - 1 : 0, prec));
  if (!b || !x) return fail(c, ALS_EINVAL, "null vector");
  MGWork& w = work_for(c, prec);
  const int l = c->L - 1;
  const size_t bytes = (size_t)(c->lev[l].g.N * c->dim) * w.es;
  begin(c);
  cudaMemcpyAsync(w.b[l], b, bytes, cudaMemcpyDeviceToDevice, c->stream);
  ALS_TRY(run_vcycle(c, w));
  cudaMemcpyAsync(x, w.x[l], bytes, cudaMemcpyDeviceToDevice, c->stream);
  return finish(c, "vcycle");
} catch (...) {
  return caught_exception();
}

als_status als_star_smooth(als_ctx* c, int level, int prec, const void* r, void* z) try {
  ALS_TRY(check_level(c, level, prec));
  if (level < 1) return fail(c, ALS_EINVAL, "the coarsest level has no smoother");
  if (!r || !z) return fail(c, ALS_EINVAL, "null vector");
  MGWork& w = work_for(c, prec);
  begin(c);
  patch_smooth(c->lev[level], prec, r, z, w.scratch[level], c->stream);
  return finish(c, "star_smooth");
} catch (...) {
  return caught_exception();
}

als_status als_prolong(als_ctx* c, int level, int prec, const void* xc, void* xf) try {
  ALS_TRY(check_level(c, level, prec));
  if (level < 1) return fail(c, ALS_EINVAL, "prolongation needs level >= 1");
  if (!xc || !xf) return fail(c, ALS_EINVAL, "null vector");
  begin(c);
  prolong_level(c, work_for(c, prec), level, xc, xf, nullptr);
  return finish(c, "prolong");
} catch (...) {
  return caught_exception();
}

als_status als_restrict(als_ctx* c, int level, int prec, const void* rf, void* rc) try {
  ALS_TRY(check_level(c, level, prec));
  if (level < 1) return fail(c, ALS_EINVAL, "restriction needs level >= 1");
  if (!rf || !rc) return fail(c, ALS_EINVAL, "null vector");
  begin(c);
  restrict_level(c, work_for(c, prec), level, rf, rc);
  return finish(c, "restrict");
} catch (...) {
  return caught_exception();
}

als_status als_coarse_solve(als_ctx* c, int prec, const void* b, void* x) try {
  ALS_TRY(check_level(c, 0, prec));
  if (!b || !x) return fail(c, ALS_EINVAL, "null vector");
  begin(c);
  coarse_apply(c->lev[0], c->coarse, prec, b, x, c->stream);
  return finish(c, "coarse_solve");
} catch (...) {
  return caught_exception();
}

als_status als_apply_stokes(als_ctx* c, const double* u, const double* p, double* yu, double* yp) try {
  if (!c || !u || !p || !yu || !yp) return c ? fail(c, ALS_EINVAL, "null vector") : ALS_EINVAL;
  const LevelDev& F = c->lev[c->L - 1];
  begin(c);
  op_apply(F, PREC_F64, OP_VISC | OP_AL | OP_BT | OP_B, c->gamma, u, yu, p, yp, c->stream);
  return finish(c, "apply_stokes");
} catch (...) {
  return caught_exception();
}

als_status als_patch_inverse(als_ctx* c, int level, long long vertex, double* out) try {
  ALS_TRY(check_level(c, level, PREC_F64));
  if (level < 1) return fail(c, ALS_EINVAL, "the coarsest level has no patches");
  const LevelDev& Lv = c->lev[level];
  if (vertex < 0 || vertex >= Lv.g.nverts) return fail(c, ALS_EINVAL, "vertex out of range");
  if (!out) return fail(c, ALS_EINVAL, "null output");
  std::vector<double> packed(Lv.pstride), full((size_t)Lv.np * Lv.np);
  if (cudaMemcpyAsync(packed.data(), Lv.inv64 + vertex * Lv.pstride, sizeof(double) * Lv.pstride,
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return cuda_check(c, "patch_inverse");
  const int np = Lv.np;
  for (int t = 0; t < np; ++t)
    for (int i = 0; i + t < np; ++i) {
      const double v = packed[diag_start(np, t) + i];
      full[(size_t)i * np + i + t] = v;
      full[(size_t)(i + t) * np + i] = v;
    }
  if (cudaMemcpy(out, full.data(), sizeof(double) * full.size(), cudaMemcpyDefault) != cudaSuccess)
    return cuda_check(c, "patch_inverse copy");
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_load_patch_inverses(als_ctx* c, int level, const double* packed) try {
  ALS_TRY(check_level(c, level, PREC_F64));
  if (level < 1) return fail(c, ALS_EINVAL, "the coarsest level has no patches");
  if (!packed) return fail(c, ALS_EINVAL, "null inverses");
  const LevelDev& Lv = c->lev[level];
  begin(c);
  if (cudaMemcpyAsync(Lv.inv64, packed, sizeof(double) * Lv.g.nverts * Lv.pstride, cudaMemcpyDefault, c->stream) !=
      cudaSuccess)
    return cuda_check(c, "load patch inverses");
  patch_derive32(Lv, c->stream);
  return finish(c, "load patch inverses");
} catch (...) {
  return caught_exception();
}

als_status als_load_coarse_inverse(als_ctx* c, const double* inv) try {
  if (!c || !inv) return c ? fail(c, ALS_EINVAL, "null inverse") : ALS_EINVAL;
  const size_t n = (size_t)c->coarse.nfree;
  begin(c);
  if (cudaMemcpyAsync(c->coarse.inv, inv, sizeof(double) * n * n, cudaMemcpyDefault, c->stream) != cudaSuccess)
    return cuda_check(c, "load coarse inverse");
  return finish(c, "load coarse inverse");
} catch (...) {
  return caught_exception();
}

als_status als_set_wait_limit(als_ctx* c, int polls) try {
  if (!c) return ALS_EINVAL;
  cudaStreamSynchronize(c->stream);
  free_graphs(c);   // the captured cycles embed the limit as a kernel argument
  for (LevelDev& Lv : c->lev) Lv.wait_polls = polls < 0 ? kWaitPolls : polls;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_solve_history(const als_ctx* c, double* out, int cap, int* count) try {
  if (!c || !count || (cap > 0 && !out)) return ALS_EINVAL;
  const std::vector<double>& h = c->run.hist;
  *count = (int)h.size();
  for (int i = 0; i < cap && i < (int)h.size(); ++i) out[i] = h[i];
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

// ---- the outer solve in stages, so that a batch can interleave the FGMRES
// iterations of several contexts (each on its own stream) with one host wait
// per round: start (inputs, lifted rhs, |b| on its way to the host), then rounds
// of launch-iteration / iteration-done, then finish.

// FGMRES (Sec. 5.1), right preconditioned, CGS2, x0 = 0, for the right-hand side in
// c->V[0]: |b| (on its way to the host), V[0] = b / |b|
static als_status fgmres_begin(als_ctx* c) {
  const cudaStream_t s = c->stream;
  const int maxit = c->opt.maxit, ldh = maxit + 1;
  double* rhs = c->V;
  vec_multidot(PREC_F64, c->n, 1, rhs, c->n, rhs, c->nrm2, c->partial, s);
  dev_init_g(maxit + 1, c->nrm2, c->g, c->beta, s);
  vec_scale_dev(PREC_F64, c->n, nullptr, c->beta, rhs, rhs, s);
  cudaMemsetAsync(c->H, 0, sizeof(double) * ldh * maxit, s);
  cudaMemcpyAsync(c->host_res + 1, c->beta, sizeof(double), cudaMemcpyDeviceToHost, s);
  return cuda_check(c, "solve rhs");
}

// queue the inputs, the lifted augmented right-hand side and |b| (no wait)
static als_status solve_start(als_ctx* c, const double* f_qp, const double* u_bc, const double* r2, double* u,
                              double* p) {
  if (!f_qp || !u || !p) return fail(c, ALS_EINVAL, "f_qp, u and p are required");
  als_ctx::SolveRun& R = c->run;
  R = als_ctx::SolveRun{};
  R.u = u;
  R.p = p;
  const int maxit = c->opt.maxit;
  ALS_TRY(alloc_solve(c, maxit));
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  const int NB = c->nq;
  begin(c);
  cudaEventCreate(&R.e0);
  cudaEventCreate(&R.e1);
  cudaEventRecord(R.e0, s);
  // inputs (host or device)
  cudaMemcpyAsync(c->f_dev, f_qp, sizeof(double) * F.g.ncells * NB * c->dim, cudaMemcpyDefault, s);
  if (u_bc) cudaMemcpyAsync(c->ubc_dev, u_bc, sizeof(double) * c->nu, cudaMemcpyDefault, s);
  else cudaMemsetAsync(c->ubc_dev, 0, sizeof(double) * c->nu, s);
  if (r2) cudaMemcpyAsync(c->r2_dev, r2, sizeof(double) * c->np, cudaMemcpyDefault, s);
  else cudaMemsetAsync(c->r2_dev, 0, sizeof(double) * c->np, s);
  ALS_TRY(cuda_check(c, "solve inputs"));
  // lifted, augmented right-hand side (Eq. (augstokessys))
  double* rhs = c->V;
  double* rhs_u = rhs;
  double* rhs_p = rhs + c->nu;
  bnd_mask(F.g, c->ubc_dev, c->uD, 1, s);                                              // u_D
  op_load_vector(F, c->f_dev, c->tu, s);                                               // F
  op_apply(F, PREC_F64, OP_VISC | OP_AL | OP_RAW, c->gamma, c->uD, c->tu2, nullptr, nullptr, s);  // A_gamma u_D
  vec_axpby(PREC_F64, c->nu, -1.0, c->tu2, 1.0, c->tu, s);                            // F - A_gamma u_D
  op_apply(F, PREC_F64, OP_B | OP_RAW, c->gamma, c->uD, nullptr, nullptr, c->tp, s);   // B u_D
  vec_axpby(PREC_F64, c->np, 1.0, c->r2_dev, -1.0, c->tp, s);                          // r2 - B u_D
  cudaMemcpyAsync(rhs_p, c->tp, sizeof(double) * c->np, cudaMemcpyDeviceToDevice, s);
  winv_scale(F.g, c->gamma, c->r2_dev, c->tp2, s, F.winv64, c->npr);                   // gamma W^-1 r2 (user part)
  op_apply(F, PREC_F64, OP_BT, c->gamma, nullptr, c->tu2, c->tp2, nullptr, s);         // B^T gamma W^-1 r2
  vec_axpby(PREC_F64, c->nu, 1.0, c->tu2, 1.0, c->tu, s);
  bnd_mask(F.g, c->tu, rhs_u, 0, s);                                                   // zero boundary rows
  return fgmres_begin(c);
}

// after the stream has drained: read |b|
static als_status solve_rhs_done(als_ctx* c) {
  als_ctx::SolveRun& R = c->run;
  ALS_TRY(check_status(c, "solve rhs"));
  R.beta = c->host_res[1];
  R.resid = R.beta;
  R.hist.assign(1, R.beta);
  R.converged = R.beta == 0.0;
  R.done = R.converged || c->opt.maxit <= 0;
  return ALS_OK;
}

// the FGMRES iteration after its preconditioner application z_k = P v_k: w = A z_k,
// Gram-Schmidt, Givens step, residual estimate on its way to the host
static void solve_iter_tail(als_ctx* c) {
  als_ctx::SolveRun& R = c->run;
  const cudaStream_t s = c->stream;
  const int k = R.k, ldh = c->opt.maxit + 1;
  double* zk = c->Z + (size_t)k * c->n;
  double* w = c->V + (size_t)(k + 1) * c->n;
  double* hcol = c->H + (size_t)k * ldh;
  matvec(c, zk, w);
  vec_multidot(PREC_F64, c->n, k + 1, c->V, c->n, w, hcol, c->partial, s);
  vec_multiaxpy(PREC_F64, c->n, k + 1, c->V, c->n, hcol, w, s, -1.0);
  vec_multidot(PREC_F64, c->n, k + 1, c->V, c->n, w, c->h2, c->partial, s);
  vec_multiaxpy_norm(PREC_F64, c->n, k + 1, c->V, c->n, c->h2, -1.0, w, c->partial, c->nrm2, s);
  vec_scale_dev(PREC_F64, c->n, nullptr, c->nrm2, w, w, s, 1);
  dev_hess_givens(k, c->H, ldh, c->h2, c->nrm2, c->cs, c->sn, c->g, c->res, s);
  cudaMemcpyAsync(c->host_res, c->res, sizeof(double), cudaMemcpyDeviceToHost, s);
}

// The mixed-mode full-factorisation preconditioner of iteration k split at its two
// FP32 cycles (the steps of precondition, in its order), so that a batch can run the
// cycles of all its instances as merged launches: phase 0 loads the first cycle's
// right-hand side, phase 1 runs between the cycles, phase 2 finishes z_k and the
// iteration.
static void precond_mixed_phase(als_ctx* c, int phase) {
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  const int k = c->run.k;
  const double* v = c->V + (size_t)k * c->n;
  double* z = c->Z + (size_t)k * c->n;
  const double* f = v;
  const double* gp = v + c->nu;
  double* x1 = z;
  double* z2 = z + c->nu;
  MGWork& w = work_for(c, PREC_F32);
  const int l = c->L - 1;
  if (phase == 0) {
    vec_cast(c->nu, f, PREC_F64, w.b[l], PREC_F32, s);
  } else if (phase == 1) {
    vec_cast(c->nu, w.x[l], PREC_F32, c->tu, PREC_F64, s);
    op_apply(F, PREC_F32, OP_B, c->gamma, w.x[l], nullptr, nullptr, c->tp32, s);     // B z1 (FP32)
    vec_cast(c->np, c->tp32, PREC_F32, c->tp, PREC_F64, s);
    vec_axpby(PREC_F64, c->np, 1.0, gp, -1.0, c->tp, s);                             // tp = g - B z1
    schur_apply(F.g.ncells, c->npr, c->schur, c->tp, z2, s);                         // z2 = -S^-1 tp
    vec_cast(c->np, z2, PREC_F64, c->tp32, PREC_F32, s);
    op_apply(F, PREC_F32, OP_BT, c->gamma, nullptr, w.b[l], c->tp32, nullptr, s);    // B^T z2 (FP32)
  } else {
    vec_cast(c->nu, w.x[l], PREC_F32, x1, PREC_F64, s);
    vec_axpby(PREC_F64, c->nu, 1.0, c->tu, -1.0, x1, s);                             // x1 = z1 - x1
    project_constant(F.g.ncells, c->npr, z2, c->partial, s);
    solve_iter_tail(c);
  }
}

// queue FGMRES iteration k (no wait); the residual estimate is on its way to the host
static als_status solve_iter_launch(als_ctx* c) {
  const int k = c->run.k;
  ALS_TRY(precondition(c, c->V + (size_t)k * c->n, c->Z + (size_t)k * c->n));
  solve_iter_tail(c);
  return ALS_OK;
}

// after the stream has drained: read the residual estimate of the iteration
static als_status solve_iter_done(als_ctx* c) {
  als_ctx::SolveRun& R = c->run;
  R.its = ++R.k;
  R.resid = c->host_res[0];
  R.hist.push_back(R.resid);
  if (!std::isfinite(R.resid)) {
    R.done = true;
    ALS_TRY(check_status(c, "fgmres"));
    return fail(c, ALS_EBREAKDOWN, "non-finite FGMRES residual");
  }
  if (R.resid <= c->opt.rtol * R.beta) R.converged = true;
  R.done = R.converged || R.k >= c->opt.maxit;
  return ALS_OK;
}

// x = Z y; u = x_u + u_D; p = x_p with zero mean; wait; report
static als_status solve_finish(als_ctx* c, als_solve_info* info) {
  als_ctx::SolveRun& R = c->run;
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  const int ldh = c->opt.maxit + 1;
  cudaMemsetAsync(c->xsol, 0, sizeof(double) * c->n, s);
  if (R.its > 0) {
    dev_backsolve(R.its, c->H, ldh, c->g, c->y, s);
    vec_multiaxpy(PREC_F64, c->n, R.its, c->Z, c->n, c->y, c->xsol, s, 1.0);
  }
  vec_axpby(PREC_F64, c->nu, 1.0, c->uD, 1.0, c->xsol, s);
  project_constant(F.g.ncells, c->npr, c->xsol + c->nu, c->partial, s);
  cudaMemcpyAsync(R.u, c->xsol, sizeof(double) * c->nu, cudaMemcpyDefault, s);
  cudaMemcpyAsync(R.p, c->xsol + c->nu, sizeof(double) * c->np, cudaMemcpyDefault, s);
  cudaEventRecord(R.e1, s);
  const als_status st = finish(c, "solve");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, R.e0, R.e1);
  cudaEventDestroy(R.e0);
  cudaEventDestroy(R.e1);
  R.e0 = R.e1 = nullptr;
  if (info) {
    info->iterations = R.its;
    info->vcycles = (c->opt.fact == ALS_FACT_FULL ? 2 : 1) * R.its;
    info->converged = R.converged ? 1 : 0;
    info->res0 = R.beta;
    info->res_final = R.resid;
    info->solve_ms = ms;
  }
  ALS_TRY(st);
  if (!R.converged) return fail(c, ALS_ENOTCONV, "FGMRES did not converge within maxit");
  return ALS_OK;
}

als_status als_solve(als_ctx* c, const double* f_qp, const double* u_bc, const double* r2, double* u, double* p,
                     als_solve_info* info) try {
  if (!c) return ALS_EINVAL;
  ALS_TRY(solve_start(c, f_qp, u_bc, r2, u, p));
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "solve rhs");
  ALS_TRY(solve_rhs_done(c));
  while (!c->run.done) {
    ALS_TRY(solve_iter_launch(c));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "fgmres");
    ALS_TRY(solve_iter_done(c));
  }
  return solve_finish(c, info);
} catch (...) {
  return caught_exception();
}


// ============================================================================
// Newton's method for the viscoplastic rheology (Sec. 5.3.1), on the GPU.
// Each step linearises at the current iterate (newton.cu: the fourth-order coefficient
// and mu at every level's Gauss points), re-runs the setup with it (als_update_coefficients),
// solves [J B^T; B 0] [du; dp] = -[R_u; R_p] (the AL-augmented, W = M_p(1/mu) form) with
// the context's FGMRES to an absolute tolerance of 1e-12 |R_0| (relative 1e-2 at most),
// and backtracks by halving until the residual norm decreases by 1e-4 alpha.  The residual
// R_u = A(mu(u)) u + B^T p - F (Dirichlet rows 0), R_p = B u is evaluated with the scalar
// viscosity mu(eps_II(u)) at the finest points.
// ============================================================================
static als_status newton_alloc(als_ctx* c) {
  als_ctx::NewtonBuf& W = c->nw;
  if (W.ready) return ALS_OK;
  const LevelDev& F = c->lev[c->L - 1];
  const int NB = c->dim == 2 ? 9 : 27, NC = c->dim == 2 ? 6 : 21;
  for (double** q : {&W.u, &W.ut, &W.du, &W.Ru, &W.F}) ALS_TRY(dalloc(c, q, c->nu));
  for (double** q : {&W.p, &W.pt, &W.dp, &W.Rp}) ALS_TRY(dalloc(c, q, c->np));
  ALS_TRY(dalloc(c, &W.mu, (size_t)F.g.ncells * NB));
  W.C.assign(c->L, nullptr);
  W.mul.assign(c->L, nullptr);
  for (int l = 0; l < c->L; ++l) {
    ALS_TRY(dalloc(c, &W.C[l], (size_t)c->lev[l].g.ncells * NB * NC));
    ALS_TRY(dalloc(c, &W.mul[l], (size_t)c->lev[l].g.ncells * NB));
  }
  W.ready = true;
  return ALS_OK;
}

// |(R_u, R_p)| at (u, p); R_u and R_p are left in c->nw
static als_status newton_residual(als_ctx* c, const als_newton_params& prm, const double* u, const double* p,
                                  double* norm) {
  als_ctx::NewtonBuf& W = c->nw;
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  newton_coeffs(F.g, F.g, u, prm.mu_ref, prm.tau_y, nullptr, W.mu, s);
  LevelDev Lm = F;                        // the finest level with the scalar viscosity mu(u)
  Lm.tensor = 0;
  Lm.ncoef = 1;
  Lm.coef64 = W.mu;
  Lm.coef32 = nullptr;
  Lm.mu64 = W.mu;
  Lm.winv64 = nullptr;
  Lm.winv32 = nullptr;
  op_apply(Lm, PREC_F64, OP_VISC | OP_BT | OP_B | OP_RAW, 0.0, u, W.Ru, p, W.Rp, s);   // A(mu) u + B^T p, B u
  vec_axpby(PREC_F64, c->nu, -1.0, W.F, 1.0, W.Ru, s);                                  // - F
  bnd_mask(F.g, W.Ru, W.Ru, 0, s);                                                      // Dirichlet rows 0
  vec_multidot(PREC_F64, c->nu, 1, W.Ru, c->nu, W.Ru, c->h2, c->partial, s);
  vec_multidot(PREC_F64, c->np, 1, W.Rp, c->np, W.Rp, c->h2 + 1, c->partial, s);
  if (cudaMemcpyAsync(c->host_res, c->h2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return cuda_check(c, "newton residual");
  *norm = std::sqrt(c->host_res[0] + c->host_res[1]);
  return ALS_OK;
}

// one FGMRES solve of the linearised system for the step (du, dp), to relative tolerance rtol
static als_status newton_step_solve(als_ctx* c, double rtol, int* its) {
  als_ctx::NewtonBuf& W = c->nw;
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  double* rhs_u = c->V;
  double* rhs_p = c->V + c->nu;
  // r2 = -R_p; rhs_u = -R_u + B^T gamma W^-1 r2 with Dirichlet rows 0
  vec_axpby(PREC_F64, c->np, -1.0, W.Rp, 0.0, rhs_p, s);
  winv_scale(F.g, c->gamma, rhs_p, c->tp2, s, F.winv64);
  op_apply(F, PREC_F64, OP_BT, c->gamma, nullptr, c->tu2, c->tp2, nullptr, s);
  vec_axpby(PREC_F64, c->nu, -1.0, W.Ru, 1.0, c->tu2, s);
  bnd_mask(F.g, c->tu2, rhs_u, 0, s);
  als_ctx::SolveRun& R = c->run;
  R = als_ctx::SolveRun{};
  R.u = W.du;
  R.p = W.dp;
  cudaEventCreate(&R.e0);
  cudaEventCreate(&R.e1);
  cudaEventRecord(R.e0, s);
  cudaMemsetAsync(c->uD, 0, sizeof(double) * c->nu, s);
  ALS_TRY(fgmres_begin(c));
  const double saved = c->opt.rtol;
  c->opt.rtol = rtol;
  als_status st = ALS_OK;
  if (cudaStreamSynchronize(s) != cudaSuccess) st = cuda_check(c, "newton step");
  if (st == ALS_OK) st = solve_rhs_done(c);
  while (st == ALS_OK && !c->run.done) {
    st = solve_iter_launch(c);
    if (st == ALS_OK && cudaStreamSynchronize(s) != cudaSuccess) st = cuda_check(c, "newton step");
    if (st == ALS_OK) st = solve_iter_done(c);
  }
  if (st == ALS_OK) st = solve_finish(c, nullptr);
  c->opt.rtol = saved;
  *its = c->run.its;
  return st;
}

extern "C" {

void als_newton_default_params(als_newton_params* prm) {
  if (!prm) return;
  prm->mu_ref = 1.0;
  prm->tau_y = 1.0;
  prm->rtol = 1e-10;
  prm->maxit = 30;
  prm->max_halvings = 12;
}

als_status als_newton_solve(als_ctx* c, const als_newton_params* prm, const double* f_qp, const double* u_bc,
                            double* u, double* p, als_newton_info* info) try {
  if (!c) return ALS_EINVAL;
  if (!prm || !f_qp || !u || !p) return fail(c, ALS_EINVAL, "parameters, f_qp, u and p are required");
  if (!c->lev[0].tensor || c->opt.schur != ALS_SCHUR_P2)
    return fail(c, ALS_EINVAL, "Newton needs a context with tensor coefficients and the P2 pairing");
  if (!(prm->mu_ref > 0.0) || !(prm->tau_y > 0.0) || !(prm->rtol > 0.0) || prm->maxit < 0 || prm->max_halvings < 0)
    return fail(c, ALS_EINVAL, "mu_ref, tau_y and rtol must be positive, maxit and max_halvings >= 0");
  ALS_TRY(alloc_solve(c, c->opt.maxit));
  ALS_TRY(newton_alloc(c));
  als_ctx::NewtonBuf& W = c->nw;
  const LevelDev& F = c->lev[c->L - 1];
  const cudaStream_t s = c->stream;
  const int NB = c->dim == 2 ? 9 : 27;
  begin(c);
  // inputs: u = u_D on the boundary, 0 inside; p = 0; the load vector F
  cudaMemcpyAsync(c->f_dev, f_qp, sizeof(double) * F.g.ncells * NB * c->dim, cudaMemcpyDefault, s);
  if (u_bc) cudaMemcpyAsync(c->ubc_dev, u_bc, sizeof(double) * c->nu, cudaMemcpyDefault, s);
  else cudaMemsetAsync(c->ubc_dev, 0, sizeof(double) * c->nu, s);
  ALS_TRY(cuda_check(c, "newton inputs"));
  bnd_mask(F.g, c->ubc_dev, W.u, 1, s);
  cudaMemsetAsync(W.p, 0, sizeof(double) * c->np, s);
  op_load_vector(F, c->f_dev, W.F, s);
  double r = 0.0;
  ALS_TRY(newton_residual(c, *prm, W.u, W.p, &r));
  W.hist.assign(1, r);
  W.lin.clear();
  int lin_total = 0;
  bool converged = r == 0.0;
  for (int k = 0; k < prm->maxit && !converged; ++k) {
    if (W.hist.back() <= prm->rtol * W.hist[0]) { converged = true; break; }
    const double eta = std::min(1e-2, std::max(1e-12, 1e-12 * W.hist[0] / W.hist.back()));
    // linearise at u: coefficients of every level, setup
    for (int l = 0; l < c->L; ++l) newton_coeffs(F.g, c->lev[l].g, W.u, prm->mu_ref, prm->tau_y, W.C[l], W.mul[l], s);
    std::vector<const double*> qp(W.C.begin(), W.C.end()), me(W.mul.begin(), W.mul.end());
    const als_coeff cf{ALS_COEFF_TENSOR, qp.data(), me.data()};
    ALS_TRY(run_setup(c, &cf));
    ALS_TRY(newton_residual(c, *prm, W.u, W.p, &r));       // R at u (for the right-hand side)
    int its = 0;
    const als_status st = newton_step_solve(c, eta, &its);
    if (st != ALS_OK && st != ALS_ENOTCONV) return st;
    W.lin.push_back(its);
    lin_total += its;
    // backtracking: halve alpha until |R| < (1 - 1e-4 alpha) |R_k|
    double alpha = 1.0, rt = 0.0;
    for (int h = 0; h < prm->max_halvings; ++h) {
      cudaMemcpyAsync(W.ut, W.u, sizeof(double) * c->nu, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(W.pt, W.p, sizeof(double) * c->np, cudaMemcpyDeviceToDevice, s);
      vec_axpby(PREC_F64, c->nu, alpha, W.du, 1.0, W.ut, s);
      vec_axpby(PREC_F64, c->np, alpha, W.dp, 1.0, W.pt, s);
      ALS_TRY(newton_residual(c, *prm, W.ut, W.pt, &rt));
      if (rt < (1.0 - 1e-4 * alpha) * W.hist.back()) break;
      alpha *= 0.5;
    }
    vec_axpby(PREC_F64, c->nu, alpha, W.du, 1.0, W.u, s);    // the step actually taken
    vec_axpby(PREC_F64, c->np, alpha, W.dp, 1.0, W.p, s);
    W.hist.push_back(rt);
  }
  if (!converged && W.hist.back() <= prm->rtol * W.hist[0]) converged = true;
  cudaMemcpyAsync(u, W.u, sizeof(double) * c->nu, cudaMemcpyDefault, s);
  cudaMemcpyAsync(p, W.p, sizeof(double) * c->np, cudaMemcpyDefault, s);
  ALS_TRY(finish(c, "newton"));
  if (info) {
    info->iterations = (int)W.hist.size() - 1;
    info->linear_iterations = lin_total;
    info->converged = converged ? 1 : 0;
    info->res0 = W.hist[0];
    info->res_final = W.hist.back();
  }
  if (!converged) return fail(c, ALS_ENOTCONV, "Newton did not reach rtol within maxit steps");
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_newton_history(const als_ctx* c, double* res, int* linear_its, int cap, int* count) try {
  if (!c || !count || (cap > 0 && (!res || !linear_its))) return ALS_EINVAL;
  const als_ctx::NewtonBuf& W = c->nw;
  *count = (int)W.hist.size();
  for (int i = 0; i < cap && i < (int)W.hist.size(); ++i) {
    res[i] = W.hist[i];
    linear_its[i] = i == 0 ? 0 : W.lin[i - 1];
  }
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

}  // extern "C"

// ============================================================================
// Batches of independent instances (uneven sizes, dimensions and parameters).
// Each instance is a full context with its own stream.  A batched solve
// interleaves the instances' FGMRES iterations: every round queues one
// iteration of every unfinished instance on its own stream and then waits once
// for all of them, so the kernels of different instances run concurrently.  The
// FP32 cycles run in one of two forms (als_batch_set_mode): merged launches, one
// per level operation for each group of instances (MergedCycle, MergedPlan above;
// in a solve each group's cycles are joined with its instances' streams by
// events), or one graph whose branches are the instances' own captured cycle
// graphs (no edges between them).
// ============================================================================
}  // extern "C"

namespace {

// ----------------------------------------------------------------------------
// Merged FP32 cycles: the V-cycles of all instances of a set, issued as one launch per
// level operation (the merged launches of batch.cuh).  The instances' hierarchies are
// aligned at the coarsest level: level index l (0 = coarsest) of the merged cycle runs
// the smoothing, transfer and GMRES operations of every instance that has a level l,
// so the coarse solves of all instances form one launch, and the sequence of
// operations each instance sees is exactly that of its own cycle_level (same kernels,
// same arithmetic, same order).  Only the patch-kernel variant of the star products and
// of the interior solves is chosen per merged operation, by merged_tune.
// ----------------------------------------------------------------------------
struct MergedCycle {
  std::vector<als_ctx*> inst;
  int Lmax = 0;
  std::vector<int> var_prod, var_int;     // per level index (>= 1)
  std::vector<float> ms_prod, ms_int;     // per level index x 3 variants (ms per launch)
  cudaGraph_t tmpl = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  bool tuned = false;
};

// why instance c cannot take part in merged cycles ("" if it can)
std::string merged_ineligible(const als_ctx* c, const als_ctx* first) {
  if (c->k != 2) return "order 3";
  if (c->lev[0].tensor) return "tensor coefficients";
  if (c->opt.store != ALS_STORE_FP32) return "bfloat16 star storage";
  if (!fused_gmres(c)) return "smoother other than GMRES(s <= 8)";
  if (c->opt.cycle != ALS_CYCLE_V) return "F-cycle";
  if (c->prof.on) return "kernel timing on";
  if (first && std::max(1, c->opt.sweeps) != std::max(1, first->opt.sweeps)) return "sweeps differ from instance 0";
  if (first && c->opt.transfer != first->opt.transfer) return "transfer differs from instance 0";
  return "";
}

void merged_free(MergedCycle& M) {
  if (M.exec) cudaGraphExecDestroy(M.exec);
  if (M.tmpl) cudaGraphDestroy(M.tmpl);
  M.exec = nullptr;
  M.tmpl = nullptr;
  M.kernels = 0;
}

// instances with a level l (l >= 0)
std::vector<als_ctx*> at_level(const MergedCycle& M, int l) {
  std::vector<als_ctx*> out;
  for (als_ctx* c : M.inst)
    if (l < c->L) out.push_back(c);
  return out;
}

// smooth_fused on level l of every instance that has it (x_is_zero: x starts at 0;
// residual: t = b - A x from the Arnoldi relation, as the pre-smoothing does)
void merged_smooth(MergedCycle& M, int l, bool x_is_zero, bool residual, cudaStream_t s) {
  const std::vector<als_ctx*> S = at_level(M, l);
  if (S.empty()) return;
  const int steps = std::max(1, S[0]->opt.sweeps);
  SmallLayout sl(steps);
  std::vector<BGmres> g;
  std::vector<BApply> ap;
  for (als_ctx* c : S) {
    MGWork& w = c->w32;
    const long long len = c->lev[l].g.N * c->dim;
    BGmres it{};
    it.n = len;
    it.b = w.b[l];
    it.Z = w.Z[l];
    it.V = w.V[l];
    it.ld = len;
    it.partial = w.partial;
    it.st = sl.dev(w.small[l]);
    it.x = w.x[l];
    it.x_zero = x_is_zero ? 1 : 0;
    it.t = residual ? w.t[l] : nullptr;
    g.push_back(it);
    ap.push_back(BApply{&c->lev[l], c->gamma, w.x[l], w.V[l],
                        ApplyEpi{w.b[l], -1.0, 0, nullptr, 0, nullptr, 1, it.st, w.partial}});
  }
  if (x_is_zero) batch_gm_start(g, s);     // V0 = b
  else batch_apply_epi(ap, s);             // V0 = b - A x
  for (int j = 0; j < steps; ++j) {
    std::vector<BPatch> prod, gath;
    std::vector<BApply> az;
    for (size_t i = 0; i < S.size(); ++i) {
      als_ctx* c = S[i];
      MGWork& w = c->w32;
      const long long len = c->lev[l].g.N * c->dim;
      void* Vj = vptr(w.V[l], w.es, (long long)j * len);
      void* Vn = vptr(w.V[l], w.es, (long long)(j + 1) * len);
      void* Zj = vptr(w.Z[l], w.es, (long long)j * len);
      const void* den = vptr(w.small[l], w.es, sl.hn + j);
      prod.push_back(BPatch{&c->lev[l], Vj, w.scratch[l], nullptr, nullptr});
      ApplyEpi e{nullptr, 1.0, j + 1, w.V[l], len, vptr(w.small[l], w.es, sl.H + (long long)j * sl.ldh), 0, g[i].st,
                 w.partial};
      if (fuse_patch_gather(c, PREC_F32)) {
        e.pout = w.scratch[l];
        e.pden = den;
      } else {
        gath.push_back(BPatch{&c->lev[l], nullptr, w.scratch[l], den, Zj});
      }
      az.push_back(BApply{&c->lev[l], c->gamma, Zj, Vn, e});
      g[i].j = j;
    }
    batch_star_products(M.var_prod[l], prod, s);    // scratch rows = A_v^-1 V_j|_v
    if (!gath.empty()) batch_patch_gather(gath, s);  // Z_j = D^-1 v_j (unfused instances)
    batch_apply_epi(az, s);                          // A Z_j, H[0..j][j]
    batch_gm_orth(g, s);                             // V_{j+1}, Givens step j
  }
  batch_gm_update(g, s);
}

void merged_restrict(MergedCycle& M, int l, cudaStream_t s) {
  const std::vector<als_ctx*> S = at_level(M, l);
  std::vector<BPatch> isv;
  std::vector<BApply> ap;
  std::vector<BTransfer> tr;
  const bool robust = S[0]->opt.transfer == ALS_TRANSFER_ROBUST;
  for (als_ctx* c : S) {
    MGWork& w = c->w32;
    isv.push_back(BPatch{&c->lev[l], w.t[l], w.t2[l], nullptr, nullptr});
    ap.push_back(BApply{&c->lev[l], c->gamma, w.t2[l], w.t3[l], ApplyEpi{}});
    tr.push_back(BTransfer{&c->lev[l - 1], &c->lev[l], w.t[l], w.b[l - 1], robust ? w.t3[l] : nullptr});
  }
  if (robust) {
    batch_interior_solve(M.var_int[l], isv, 0, s);   // t2 = sum_K E_K A_K^-1 E_K^T t
    batch_apply_al(ap, s);                           // t3 = G t2
  }
  batch_restrict(tr, s);                             // b_{l-1} = P_H^T (t - t3)
}

void merged_prolong(MergedCycle& M, int l, cudaStream_t s) {
  const std::vector<als_ctx*> S = at_level(M, l);
  std::vector<BPatch> isv;
  std::vector<BApply> ap;
  std::vector<BTransfer> tr;
  const bool robust = S[0]->opt.transfer == ALS_TRANSFER_ROBUST;
  for (als_ctx* c : S) {
    MGWork& w = c->w32;
    tr.push_back(BTransfer{&c->lev[l - 1], &c->lev[l], w.x[l - 1], w.t[l], w.x[l]});
    ap.push_back(BApply{&c->lev[l], c->gamma, w.t[l], w.t3[l], ApplyEpi{}});
    isv.push_back(BPatch{&c->lev[l], w.t3[l], w.x[l], nullptr, nullptr});
  }
  batch_prolong(tr, s);                              // t = P_H x_{l-1}, x += t
  if (robust) {
    batch_apply_al(ap, s);                           // t3 = G t
    batch_interior_solve(M.var_int[l], isv, 1, s);   // x -= sum_K E_K A_K^-1 E_K^T t3
  }
}

// one merged V-cycle: w32.b[L-1] -> w32.x[L-1] of every instance
void merged_cycle(MergedCycle& M, cudaStream_t s) {
  for (int l = M.Lmax - 1; l >= 1; --l) {
    merged_smooth(M, l, true, true, s);
    merged_restrict(M, l, s);
  }
  std::vector<BCoarse> co;
  for (als_ctx* c : M.inst) co.push_back(BCoarse{&c->lev[0], &c->coarse, c->w32.b[0], c->w32.x[0]});
  batch_coarse_apply(co, s);
  for (int l = 1; l < M.Lmax; ++l) {
    merged_prolong(M, l, s);
    merged_smooth(M, l, false, false, s);
  }
}

// Autotuner of the merged cycle: for every level index, time the three patch-kernel
// variants of the merged star products and of the merged interior solves (one warm-up
// and three timed launches each, CUDA events) and keep the fastest.  Inputs: the
// instances' zeroed V_0 of that level; outputs go to scratch the cycle overwrites.
void merged_tune(MergedCycle& M, cudaStream_t s) {
  const long long launches0 = launch_count();
  M.var_prod.assign(M.Lmax, 0);
  M.var_int.assign(M.Lmax, 0);
  M.ms_prod.assign(3 * M.Lmax, 0.f);
  M.ms_int.assign(3 * M.Lmax, 0.f);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int l = 1; l < M.Lmax; ++l) {
    std::vector<BPatch> prod, isv;
    for (als_ctx* c : at_level(M, l)) {
      MGWork& w = c->w32;
      vec_zero(PREC_F32, c->lev[l].g.N * c->dim, w.V[l], s);
      prod.push_back(BPatch{&c->lev[l], w.V[l], w.scratch[l], nullptr, nullptr});
      isv.push_back(BPatch{&c->lev[l], w.V[l], w.t2[l], nullptr, nullptr});
    }
    for (int kind = 0; kind < 2; ++kind) {
      float best = 1e30f;
      for (int v = 0; v < 3; ++v) {
        for (int rep = 0; rep < 4; ++rep) {
          if (rep == 1) cudaEventRecord(e0, s);
          if (kind == 0) batch_star_products(v, prod, s);
          else batch_interior_solve(v, isv, 1, s);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.f;
        (kind == 0 ? M.ms_prod : M.ms_int)[3 * l + v] = ms;
        if (ms < best) {
          best = ms;
          (kind == 0 ? M.var_prod : M.var_int)[l] = v;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  count_launch(-(launch_count() - launches0));   // tuning launches are not work of a step
  M.tuned = true;
}

// capture the merged cycle (tuning first, once) and instantiate it
als_status merged_build(MergedCycle& M, cudaStream_t s, std::string& err) {
  if (M.exec) return ALS_OK;
  M.Lmax = 0;
  for (als_ctx* c : M.inst) M.Lmax = std::max(M.Lmax, c->L);
  static bool prepared = false;
  if (!prepared) {
    batch_patch_prepare();
    batch_coarse_prepare();
    prepared = true;
  }
  if (!M.tuned) merged_tune(M, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    err = std::string("merged cycle tuning: ") + cudaGetErrorString(cudaGetLastError());
    return ALS_ECUDA;
  }
  const long long c0 = launch_count();
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    err = "merged cycle: begin capture";
    cudaGetLastError();
    return ALS_ECUDA;
  }
  merged_cycle(M, s);
  const cudaError_t ec = cudaStreamEndCapture(s, &M.tmpl);
  M.kernels = launch_count() - c0;
  count_launch(-M.kernels);
  if (ec != cudaSuccess || cudaGraphInstantiate(&M.exec, M.tmpl, 0) != cudaSuccess) {
    err = std::string("merged cycle: capture/instantiate: ") + cudaGetErrorString(cudaGetLastError());
    merged_free(M);
    return ALS_ECUDA;
  }
  return ALS_OK;
}

// A plan of merged cycles: the instances split into groups, each group's cycles merged
// (one launch per level operation for the group), the groups' captured cycles run as
// independent branches of one graph, so that one group's latency-bound levels overlap
// another's bandwidth-bound ones.  Groupings: 0 = one group, 1 = by dimension, 2 = by
// dimension and level count, 3 = by shape (dimension, cells, levels), 4 = by shape in
// chunks of at most four instances.
constexpr int kGroupings = 5;
struct MergedPlan {
  int grouping = -1;
  std::vector<MergedCycle> g;
  cudaGraph_t tmpl = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
};

std::vector<std::vector<int>> plan_groups(const std::vector<als_ctx*>& inst, int grouping) {
  std::vector<std::vector<int>> out;
  std::vector<long long> keys;
  std::vector<int> fill;   // grouping 4: members of the current chunk of each shape
  for (int i = 0; i < (int)inst.size(); ++i) {
    const als_ctx* c = inst[i];
    const long long shape = (100LL * c->dim + c->L) * 100000LL + c->lev[c->L - 1].g.n[0];
    long long key = 0;
    if (grouping == 1) key = c->dim;
    else if (grouping == 2) key = 100LL * c->dim + c->L;
    else if (grouping >= 3) key = shape;
    size_t k = keys.size();
    for (size_t q = 0; q < keys.size(); ++q)
      if (keys[q] == key && (grouping != 4 || fill[q] < 4)) { k = q; break; }
    if (k == keys.size()) {
      keys.push_back(key);
      fill.push_back(0);
      out.emplace_back();
    }
    out[k].push_back(i);
    ++fill[k];
  }
  return out;
}

void plan_free(MergedPlan& P) {
  for (MergedCycle& M : P.g) merged_free(M);
  P.g.clear();
  if (P.exec) cudaGraphExecDestroy(P.exec);
  if (P.tmpl) cudaGraphDestroy(P.tmpl);
  P.exec = nullptr;
  P.tmpl = nullptr;
  P.kernels = 0;
  P.grouping = -1;
}

// build (tune, capture) every group of a grouping and the graph of their branches
als_status plan_build(MergedPlan& P, const std::vector<als_ctx*>& inst, int grouping, cudaStream_t s,
                      std::string& err) {
  plan_free(P);
  P.grouping = grouping;
  for (const std::vector<int>& grp : plan_groups(inst, grouping)) {
    P.g.emplace_back();
    for (int i : grp) P.g.back().inst.push_back(inst[i]);
  }
  for (MergedCycle& M : P.g) ALS_TRY(merged_build(M, s, err));
  if (cudaGraphCreate(&P.tmpl, 0) != cudaSuccess) {
    err = "merged plan: graph create";
    cudaGetLastError();
    return ALS_ECUDA;
  }
  for (MergedCycle& M : P.g) {
    cudaGraphNode_t node;
    if (cudaGraphAddChildGraphNode(&node, P.tmpl, nullptr, 0, M.tmpl) != cudaSuccess) {
      err = "merged plan: child graph node";
      cudaGetLastError();
      return ALS_ECUDA;
    }
    P.kernels += M.kernels;
  }
  if (cudaGraphInstantiate(&P.exec, P.tmpl, 0) != cudaSuccess) {
    err = "merged plan: graph instantiate";
    cudaGetLastError();
    P.exec = nullptr;
    return ALS_ECUDA;
  }
  return ALS_OK;
}

}  // namespace

struct als_batch {
  std::vector<als_ctx*> ctx;
  cudaStream_t user_stream = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::string err;
  int mode = ALS_BATCH_BRANCHES;
  MergedPlan plan;                   // every instance (als_batch_vcycle), grouping chosen by time
  int forced_grouping = -1;          // als_batch_set_grouping: a fixed grouping, -1 = tuned
  float plan_ms[kGroupings] = {-1.f, -1.f, -1.f, -1.f, -1.f};   // measured cycle time of each grouping
  std::vector<MergedCycle> live;     // per group of the plan: its unfinished instances (solves)
  std::vector<cudaEvent_t> ev;       // per instance: joins of the merged cycles of a solve
  std::vector<cudaEvent_t> gev;      // per group
  std::vector<cudaStream_t> gs;      // per group: where its merged cycles run
  cudaStream_t mstream = nullptr;    // where the plan's graph runs
};

// streams and events of the merged cycles (created on first use)
static als_status batch_merged_init(als_batch* b) {
  if (b->mstream) return ALS_OK;
  if (cudaStreamCreateWithFlags(&b->mstream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    b->mstream = nullptr;
    b->err = "batch stream creation failed";
    return ALS_ECUDA;
  }
  b->ev.assign(b->ctx.size(), nullptr);
  for (cudaEvent_t& e : b->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return ALS_OK;
}

// The plan of the batch's merged cycles (first use): every grouping that gives a new
// partition is built and timed over three cycles (CUDA events, after one warm-up
// cycle) on the instances' current right-hand sides, and the fastest is kept.
static als_status batch_plan(als_batch* b) {
  if (b->plan.exec) return ALS_OK;
  ALS_TRY(batch_merged_init(b));
  const cudaStream_t s = b->mstream;
  static bool prepared = false;
  if (!prepared) {
    batch_patch_prepare();
    batch_coarse_prepare();
    prepared = true;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<std::vector<std::vector<int>>> seen;
  float best = 1e30f;
  int best_g = 0;
  for (int grouping = 0; grouping < kGroupings; ++grouping) {
    if (b->forced_grouping >= 0 && grouping != b->forced_grouping) continue;
    const std::vector<std::vector<int>> part = plan_groups(b->ctx, grouping);
    if (std::find(seen.begin(), seen.end(), part) != seen.end()) continue;   // the same partition
    seen.push_back(part);
    MergedPlan P;
    als_status st = plan_build(P, b->ctx, grouping, s, b->err);
    if (st == ALS_OK) {
      for (int rep = 0; rep < 4; ++rep) {
        if (rep == 1) cudaEventRecord(e0, s);
        if (cudaGraphLaunch(P.exec, s) != cudaSuccess) st = ALS_ECUDA;
      }
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = ALS_ECUDA;
    }
    if (st != ALS_OK) {
      plan_free(P);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (b->err.empty()) b->err = "merged plan tuning failed";
      return st == ALS_OK ? ALS_ECUDA : st;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->plan_ms[grouping] = ms / 3.f;
    if (ms < best) {
      best = ms;
      best_g = grouping;
    }
    plan_free(P);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ALS_TRY(plan_build(b->plan, b->ctx, best_g, s, b->err));
  b->gev.assign(b->plan.g.size(), nullptr);
  b->gs.assign(b->plan.g.size(), nullptr);
  for (size_t k = 0; k < b->plan.g.size(); ++k) {
    cudaEventCreateWithFlags(&b->gev[k], cudaEventDisableTiming);
    if (cudaStreamCreateWithFlags(&b->gs[k], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      b->err = "batch stream creation failed";
      return ALS_ECUDA;
    }
  }
  b->live.assign(b->plan.g.size(), MergedCycle{});
  return ALS_OK;
}

static als_status batch_fail(als_batch* b, als_status code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

extern "C" {

als_status als_batch_create(int count, const als_mesh* meshes, const als_coeff* coeffs, const double* gammas,
                            const als_options* opts, void* stream, als_batch** out) try {
  if (!out) return ALS_EINVAL;
  *out = nullptr;
  if (count < 1 || !meshes || !coeffs || !gammas) {
    t_create_err = "empty batch or null arrays";
    return ALS_EINVAL;
  }
  als_batch* b = new als_batch;
  b->user_stream = (cudaStream_t)stream;
  for (int i = 0; i < count; ++i) {
    als_ctx* c = nullptr;
    const als_status st = als_create(&meshes[i], &coeffs[i], gammas[i], opts ? &opts[i] : nullptr, stream, &c);
    if (st != ALS_OK) {
      t_create_err = "instance " + std::to_string(i) + ": " + t_create_err;
      for (als_ctx* d : b->ctx) als_destroy(d);
      delete b;
      return st;
    }
    b->ctx.push_back(c);
  }
  bool all = true;
  for (als_ctx* c : b->ctx) all = all && merged_ineligible(c, b->ctx[0]).empty();
  b->mode = all ? ALS_BATCH_MERGED : ALS_BATCH_BRANCHES;
  *out = b;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_destroy(als_batch* b) try {
  if (!b) return ALS_EINVAL;
  for (als_ctx* c : b->ctx) cudaStreamSynchronize(c->stream);
  if (b->mstream) cudaStreamSynchronize(b->mstream);
  for (int k = 0; k < 2; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
  }
  for (cudaStream_t gs : b->gs)
    if (gs) cudaStreamSynchronize(gs);
  plan_free(b->plan);
  for (MergedCycle& M : b->live) merged_free(M);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : b->gev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t gs : b->gs)
    if (gs) cudaStreamDestroy(gs);
  if (b->mstream) cudaStreamDestroy(b->mstream);
  for (als_ctx* c : b->ctx) als_destroy(c);
  delete b;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_context(als_batch* b, int i, als_ctx** ctx) try {
  if (!b || !ctx) return ALS_EINVAL;
  if (i < 0 || i >= (int)b->ctx.size()) return batch_fail(b, ALS_EINVAL, "instance index out of range");
  *ctx = b->ctx[i];
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_solve(als_batch* b, const double* const* f_qp, const double* const* u_bc,
                           const double* const* r2, double* const* u, double* const* p, als_solve_info* infos) try {
  if (!b || !f_qp || !u || !p) return ALS_EINVAL;
  const int n = (int)b->ctx.size();
  std::vector<als_status> st(n, ALS_OK);
  std::vector<bool> live(n, false);
  for (int i = 0; i < n; ++i) {
    st[i] = solve_start(b->ctx[i], f_qp[i], u_bc ? u_bc[i] : nullptr, r2 ? r2[i] : nullptr, u[i], p[i]);
    live[i] = st[i] == ALS_OK;
  }
  for (int i = 0; i < n; ++i) {
    if (!live[i]) continue;
    if (cudaStreamSynchronize(b->ctx[i]->stream) != cudaSuccess) st[i] = cuda_check(b->ctx[i], "solve rhs");
    else st[i] = solve_rhs_done(b->ctx[i]);
    live[i] = st[i] == ALS_OK;
  }
  // merged cycles: every instance mixed, with the full block factorisation (two cycles
  // per preconditioner application, see precond_mixed_phase)
  bool merged = b->mode == ALS_BATCH_MERGED;
  for (als_ctx* c : b->ctx) merged = merged && c->opt.mode == ALS_MODE_MIXED && c->opt.fact == ALS_FACT_FULL;
  std::vector<MergedCycle*> cur;   // per group: the graph its cycles run in (the plan's, at first)
  if (merged) {
    const als_status ps = batch_plan(b);
    if (ps != ALS_OK) return ps;
    for (MergedCycle& F : b->plan.g) cur.push_back(&F);
  }
  for (;;) {
    bool any = false;
    if (merged) {
      // per group of the plan: its unfinished instances' two merged cycles, on the
      // group's stream, joined with those instances' own streams by events
      for (size_t k = 0; k < b->plan.g.size(); ++k) {
        std::vector<als_ctx*> set;
        std::vector<int> act;
        for (als_ctx* c : b->plan.g[k].inst) {
          const int i = (int)(std::find(b->ctx.begin(), b->ctx.end(), c) - b->ctx.begin());
          if (live[i] && !c->run.done) {
            set.push_back(c);
            act.push_back(i);
          }
        }
        if (set.empty()) continue;
        // The group's graph is re-captured for its unfinished instances only once the
        // finished ones it still cycles (their results unused) hold more than a quarter
        // of its fine-level unknowns: capture and instantiation cost milliseconds, and
        // instances finish one by one.  The group's tuning serves every subset of it.
        long long all = 0, done = 0;
        for (als_ctx* c : cur[k]->inst) {
          const long long w = c->lev[c->L - 1].g.N;
          all += w;
          if (std::find(set.begin(), set.end(), c) == set.end()) done += w;
        }
        const cudaStream_t gs = b->gs[k];
        if (4 * done > all) {
          MergedCycle& M = b->live[k];
          merged_free(M);
          M.inst = set;
          M.var_prod = b->plan.g[k].var_prod;
          M.var_int = b->plan.g[k].var_int;
          M.tuned = true;
          const als_status bs = merged_build(M, gs, b->err);
          if (bs != ALS_OK) return bs;
          cur[k] = &M;
        }
        const MergedCycle& M = *cur[k];
        for (int phase = 0; phase < 2; ++phase) {
          for (int i : act) {
            als_ctx* c = b->ctx[i];
            if (phase > 0) cudaStreamWaitEvent(c->stream, b->gev[k], 0);
            precond_mixed_phase(c, phase);
            cudaEventRecord(b->ev[i], c->stream);
            cudaStreamWaitEvent(gs, b->ev[i], 0);
          }
          if (cudaGraphLaunch(M.exec, gs) != cudaSuccess) return batch_fail(b, ALS_ECUDA, "merged cycle launch");
          count_launch(M.kernels);
          cudaEventRecord(b->gev[k], gs);
        }
        for (int i : act) {
          als_ctx* c = b->ctx[i];
          cudaStreamWaitEvent(c->stream, b->gev[k], 0);
          precond_mixed_phase(c, 2);
        }
        any = true;
      }
    } else {
      for (int i = 0; i < n; ++i) {
        if (!live[i] || b->ctx[i]->run.done) continue;
        st[i] = solve_iter_launch(b->ctx[i]);
        if (st[i] != ALS_OK) live[i] = false;
        else any = true;
      }
    }
    if (!any) break;
    for (int i = 0; i < n; ++i) {
      if (!live[i] || b->ctx[i]->run.done) continue;
      if (cudaStreamSynchronize(b->ctx[i]->stream) != cudaSuccess) st[i] = cuda_check(b->ctx[i], "fgmres");
      else st[i] = solve_iter_done(b->ctx[i]);
      if (st[i] != ALS_OK) live[i] = false;
    }
  }
  als_status first = ALS_OK;
  for (int i = 0; i < n; ++i) {
    if (live[i]) st[i] = solve_finish(b->ctx[i], infos ? &infos[i] : nullptr);
    else if (infos) infos[i] = als_solve_info{b->ctx[i]->run.its, 0, 0, b->ctx[i]->run.beta, b->ctx[i]->run.resid, 0.0};
    if (st[i] != ALS_OK && first == ALS_OK) {
      first = st[i];
      b->err = "instance " + std::to_string(i) + ": " + b->ctx[i]->err;
    }
  }
  return first;
} catch (...) {
  return caught_exception();
}

als_status als_batch_vcycle(als_batch* b, int prec, const void* const* bv, void* const* xv) try {
  if (!b || !bv || !xv) return ALS_EINVAL;
  if (prec != PREC_F64 && prec != PREC_F32) return batch_fail(b, ALS_EINVAL, "prec must be FP64 or FP32");
  const int n = (int)b->ctx.size();
  const int k = prec == PREC_F64 ? 0 : 1;
  for (int i = 0; i < n; ++i)
    if (!bv[i] || !xv[i]) return batch_fail(b, ALS_EINVAL, "null vector");
  if (prec == PREC_F32 && b->mode == ALS_BATCH_MERGED) {
    // one merged launch per level operation for all instances
    ALS_TRY(batch_merged_init(b));
    for (int i = 0; i < n; ++i) cudaStreamSynchronize(b->ctx[i]->stream);
    const cudaStream_t s = b->mstream;
    cudaEventRecord(b->ctx[0]->order_ev, b->user_stream);
    cudaStreamWaitEvent(s, b->ctx[0]->order_ev, 0);
    for (int i = 0; i < n; ++i) {
      als_ctx* c = b->ctx[i];
      const int l = c->L - 1;
      cudaMemcpyAsync(c->w32.b[l], bv[i], (size_t)(c->lev[l].g.N * c->dim) * 4, cudaMemcpyDeviceToDevice, s);
    }
    const als_status st = batch_plan(b);   // first call: groupings built and timed (the cycle reads b only)
    if (st != ALS_OK) return st;
    if (cudaGraphLaunch(b->plan.exec, s) != cudaSuccess) return batch_fail(b, ALS_ECUDA, "merged cycle launch");
    count_launch(b->plan.kernels);
    for (int i = 0; i < n; ++i) {
      als_ctx* c = b->ctx[i];
      const int l = c->L - 1;
      cudaMemcpyAsync(xv[i], c->w32.x[l], (size_t)(c->lev[l].g.N * c->dim) * 4, cudaMemcpyDeviceToDevice, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      const cudaError_t e = cudaGetLastError();
      return batch_fail(b, ALS_ECUDA, std::string("merged cycle: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < n; ++i) {
      const als_status cs = check_status(b->ctx[i], "merged cycle");
      if (cs != ALS_OK) return batch_fail(b, cs, "instance " + std::to_string(i) + ": " + b->ctx[i]->err);
    }
    return ALS_OK;
  }
  if (!b->exec[k]) {
    // one graph: the instances' captured cycle graphs as independent child graphs
    auto drop = [&](als_status st, const std::string& msg) {
      if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
      b->graph[k] = nullptr;
      cudaGetLastError();
      return batch_fail(b, st, msg);
    };
    if (cudaGraphCreate(&b->graph[k], 0) != cudaSuccess) return drop(ALS_ECUDA, "graph create");
    for (int i = 0; i < n; ++i) {
      als_ctx* c = b->ctx[i];
      if (c->prof.on || !c->use_graph)
        return drop(ALS_EINVAL, "batched cycles need graph capture and profiling off");
      MGWork& w = work_for(c, prec);
      const als_status st = ensure_graph(c, w);
      if (st != ALS_OK) return drop(st, c->err);
      cudaGraphNode_t node;
      if (cudaGraphAddChildGraphNode(&node, b->graph[k], nullptr, 0, w.graph_tmpl) != cudaSuccess)
        return drop(ALS_ECUDA, "child graph node");
    }
    if (cudaGraphInstantiate(&b->exec[k], b->graph[k], 0) != cudaSuccess) {
      b->exec[k] = nullptr;
      return drop(ALS_ECUDA, "batch graph instantiate");
    }
  }
  // the instances' streams must be idle: their buffers are the graph's
  for (int i = 0; i < n; ++i) cudaStreamSynchronize(b->ctx[i]->stream);
  const cudaStream_t s = b->ctx[0]->stream;
  cudaEvent_t ev = b->ctx[0]->order_ev;
  cudaEventRecord(ev, b->user_stream);
  cudaStreamWaitEvent(s, ev, 0);
  for (int i = 0; i < n; ++i) {
    als_ctx* c = b->ctx[i];
    MGWork& w = work_for(c, prec);
    const int l = c->L - 1;
    if (!bv[i] || !xv[i]) return batch_fail(b, ALS_EINVAL, "null vector");
    cudaMemcpyAsync(w.b[l], bv[i], (size_t)(c->lev[l].g.N * c->dim) * w.es, cudaMemcpyDeviceToDevice, s);
  }
  if (cudaGraphLaunch(b->exec[k], s) != cudaSuccess) return batch_fail(b, ALS_ECUDA, "batch graph launch");
  long long kernels = 0;
  for (int i = 0; i < n; ++i) {
    als_ctx* c = b->ctx[i];
    MGWork& w = work_for(c, prec);
    const int l = c->L - 1;
    kernels += w.graph_kernels;
    cudaMemcpyAsync(xv[i], w.x[l], (size_t)(c->lev[l].g.N * c->dim) * w.es, cudaMemcpyDeviceToDevice, s);
  }
  count_launch(kernels);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return batch_fail(b, ALS_ECUDA, std::string("batch cycle: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < n; ++i) {
    const als_status st = check_status(b->ctx[i], "batch cycle");
    if (st != ALS_OK) return batch_fail(b, st, b->ctx[i]->err);
  }
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

const char* als_batch_last_error(const als_batch* b) { return b ? b->err.c_str() : "null batch"; }

als_status als_batch_set_mode(als_batch* b, int mode) try {
  if (!b) return ALS_EINVAL;
  if (mode != ALS_BATCH_MERGED && mode != ALS_BATCH_BRANCHES) return batch_fail(b, ALS_EINVAL, "unknown batch mode");
  if (mode == ALS_BATCH_MERGED)
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      const std::string why = merged_ineligible(b->ctx[i], b->ctx[0]);
      if (!why.empty())
        return batch_fail(b, ALS_EINVAL, "instance " + std::to_string(i) + " cannot run merged cycles: " + why);
    }
  b->mode = mode;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_set_grouping(als_batch* b, int grouping) try {
  if (!b) return ALS_EINVAL;
  if (grouping < -1 || grouping >= kGroupings) return batch_fail(b, ALS_EINVAL, "grouping must be -1 .. 4");
  for (als_ctx* c : b->ctx) cudaStreamSynchronize(c->stream);
  for (cudaStream_t gs : b->gs)
    if (gs) cudaStreamSynchronize(gs);
  if (b->mstream) cudaStreamSynchronize(b->mstream);
  plan_free(b->plan);
  for (MergedCycle& M : b->live) merged_free(M);
  b->live.clear();
  for (cudaEvent_t e : b->gev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t gs : b->gs)
    if (gs) cudaStreamDestroy(gs);
  b->gev.clear();
  b->gs.clear();
  for (float& t : b->plan_ms) t = -1.f;
  b->forced_grouping = grouping;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_get_mode(const als_batch* b, int* mode) try {
  if (!b || !mode) return ALS_EINVAL;
  *mode = b->mode;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_merged_plan(const als_batch* b, int* grouping, int* groups, float* ms, long long* kernels) try {
  if (!b || !grouping || !groups) return ALS_EINVAL;
  if (!b->plan.exec) return ALS_EINVAL;
  *grouping = b->plan.grouping;
  *groups = (int)b->plan.g.size();
  if (ms)
    for (int k = 0; k < kGroupings; ++k) ms[k] = b->plan_ms[k];
  if (kernels) *kernels = b->plan.kernels;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_batch_merged_tune(const als_batch* b, int group, int level, int* products_variant,
                                 int* interior_variant, float* ms, int* instances) try {
  if (!b || !products_variant || !interior_variant) return ALS_EINVAL;
  if (!b->plan.exec || group < 0 || group >= (int)b->plan.g.size()) return ALS_EINVAL;
  const MergedCycle& M = b->plan.g[group];
  if (level < 1 || level >= M.Lmax) return ALS_EINVAL;
  *products_variant = M.var_prod[level];
  *interior_variant = M.var_int[level];
  if (ms)
    for (int v = 0; v < 3; ++v) {
      ms[v] = M.ms_prod[3 * level + v];
      ms[3 + v] = M.ms_int[3 * level + v];
    }
  if (instances)
    for (size_t i = 0; i < M.inst.size(); ++i)
      instances[i] = (int)(std::find(b->ctx.begin(), b->ctx.end(), M.inst[i]) - b->ctx.begin());
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_set_patch_kernel(als_ctx* c, int level, int variant) try {
  if (!c) return ALS_EINVAL;
  if (level < 1 || level >= c->L) return fail(c, ALS_EINVAL, "level must be in [1, levels)");
  if (variant < -1 || variant > 2) return fail(c, ALS_EINVAL, "variant must be -1, 0, 1 or 2");
  cudaStreamSynchronize(c->stream);
  free_graphs(c);   // the captured cycles embed the variant
  c->lev[level].patch_kernel = variant;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

als_status als_autotune_info(als_ctx* c, int level, int* variant, float* ms) try {
  if (!c || !variant) return c ? fail(c, ALS_EINVAL, "null output") : ALS_EINVAL;
  if (level < 1 || level >= c->L) return fail(c, ALS_EINVAL, "level must be in [1, levels)");
  const LevelDev& Lv = c->lev[level];
  *variant = Lv.patch_kernel;
  if (ms)
    for (int k = 0; k < 3; ++k) ms[k] = Lv.patch_kernel >= 0 ? Lv.tune_ms[k] : 0.f;
  return ALS_OK;
} catch (...) {
  return caught_exception();
}

}  // extern "C"
