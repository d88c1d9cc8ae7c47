/*
 * alstokes.h - C ABI of a GB300 (sm_103a) implementation of the gamma-robust
 * augmented-Lagrangian multigrid solver for variable-viscosity Stokes flow of
 * Shih, Stadler & Wechsung, "Robust multigrid techniques for augmented
 * Lagrangian preconditioning of incompressible Stokes equations with extreme
 * viscosity variations" (arXiv 2107.00820).
 *
 * Discretisation: [Q2]^d x P1^disc (d = 2, 3) on a uniform quad/hex mesh of the
 * unit box (0,1)^d with n[k] cells per direction, homogeneous structure on
 * every multigrid level (level 0 = coarsest, level L-1 = finest, n_l = n / 2^(L-1-l)).
 *
 * Data layout (all arrays dense, C order, no padding; for options.order = 3 the
 * counts change as its documentation states: N = prod(3 n_k + 1), 4^d points and
 * C(d + 2, d) pressure coefficients per cell):
 *   velocity vector : d blocks of N nodal values, N = prod(2 n_k + 1), node
 *                     index x-fastest; Dirichlet (boundary) entries are kept
 *                     and carry identity rows.
 *   pressure vector : [cell][d+1] coefficients of {1, xi_0, .., xi_(d-1)} on the
 *                     reference cell [-1,1]^d, cell index x-fastest.
 *   point data      : [cell][3^d] at the 3-point Gauss-Legendre points of each
 *                     cell (point index x-fastest), optionally [..][m] with
 *                     m = 3 (2D vector), 6 / 21 (Mandel tensor, upper triangle
 *                     row-major; components (e00,e11,sqrt2 e01) in 2D and
 *                     (e00,e11,e22,sqrt2 e12,sqrt2 e02,sqrt2 e01) in 3D).
 *
 * Ownership: array arguments of als_create and als_solve may be host or
 * device pointers (copied with cudaMemcpyDefault); vectors passed to
 * als_apply_agamma, als_vcycle and the stage entry points are caller-owned
 * DEVICE pointers of the stated precision, valid for the duration of the
 * call.  The context owns every internal buffer and frees it in als_destroy.
 * The context runs its kernels on an internal stream that is ordered after
 * the work already queued on the stream given to als_create; every call
 * returns after its own work has finished.  A context is not thread-safe.
 *
 * Errors: every call returns an als_status; no exception crosses the ABI.
 * Device-side failures (a non-positive pivot, a Krylov breakdown) are
 * recorded on the device and reported by the call that finishes the work;
 * als_last_error() returns a message.  A failed als_create leaves *out NULL.
 *
 * Launch switches read once per process from the environment (results do not
 * depend on them unless stated): ALS_NO_GRAPH=1 issues every cycle kernel by
 * kernel instead of replaying a captured CUDA graph; ALS_PDL=0 launches without
 * programmatic dependent launch; ALS_PATCH_KERNEL=tma2|tma3|direct forces one FP32
 * star-patch kernel variant on every level; ALS_FUSE_GATHER=0 keeps the separate
 * patch-gather kernel in the FP32 3D smoother (bitwise the same results);
 * ALS_SPLIT_STARS=1 / 0 makes every smoothed level store its FP32 star inverses split
 * (interior stars block-packed, boundary stars restricted to their free dofs, applied by a
 * second kernel) or whole (every star padded to d 3^d dofs); by default levels with at
 * least 32768 vertices are split (the FP32 results differ in the rounding of the boundary
 * stars' sums).
 */
#ifndef ALSTOKES_H
#define ALSTOKES_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct als_ctx als_ctx;

typedef enum {
  ALS_OK = 0,
  ALS_EINVAL = 1,      /* invalid argument (sizes, levels, options, NULL) */
  ALS_ENOMEM = 2,      /* device or host allocation failed (no C++ exception crosses this ABI) */
  ALS_ECUDA = 3,       /* a CUDA runtime call failed */
  ALS_ENOTSPD = 4,     /* non-positive pivot in the symmetric sweep of a patch or the coarse operator */
  ALS_ENOTCONV = 5,    /* FGMRES did not reach rtol within maxit iterations */
  ALS_EBREAKDOWN = 6,  /* Krylov breakdown or a non-finite residual */
  ALS_ETIMEOUT = 7     /* a bounded device-side wait gave up: the FP32 star-smoother kernel's wait
                          for its inverse blocks (als_set_wait_limit); the kernel records it, waits
                          for its own copies in flight and returns, the context stays usable */
} als_status;

enum { ALS_COEFF_SCALAR = 0, ALS_COEFF_TENSOR = 1 };
enum { ALS_PREC_FP64 = 0, ALS_PREC_FP32 = 1 };
enum { ALS_MODE_FP64 = 0, ALS_MODE_MIXED = 1 };
enum { ALS_SMOOTH_GMRES = 0, ALS_SMOOTH_RICHARDSON = 1 };
enum { ALS_TRANSFER_ROBUST = 0, ALS_TRANSFER_STANDARD = 1 };
enum { ALS_SCHUR_P1 = 0, ALS_SCHUR_P2 = 1 };
enum { ALS_CYCLE_V = 0, ALS_CYCLE_F = 1 };
enum { ALS_FACT_FULL = 0, ALS_FACT_UPPER = 1, ALS_FACT_LOWER = 2, ALS_FACT_DIAG = 3 };
enum { ALS_SETUP_AUTO = 0, ALS_SETUP_FP64 = 1 };
enum { ALS_STORE_FP32 = 0, ALS_STORE_BF16 = 1 };

/* Unit box (0,1)^dim with n[k] cells per direction on the finest level;
 * n[k] must be divisible by 2^(levels-1) and the coarsest level must have
 * at least 2 cells per direction.  n[2] is ignored for dim = 2. */
typedef struct {
  int dim;
  int n[3];
  int levels;
} als_mesh;

/* Viscosity at the Gauss points of every level (rediscretisation on each
 * level, Sec. 5.1).  SCALAR: qp[l] is [cell][3^d] mu.  TENSOR: qp[l] is
 * [cell][3^d][6|21] Mandel C (Eq. (stokes-lin)) and mu_eff[l] is the
 * [cell][3^d] scalar used by the Schur-complement approximation. */
typedef struct {
  int kind;
  const double* const* qp;
  const double* const* mu_eff;
} als_coeff;

typedef struct {
  int smoother;   /* ALS_SMOOTH_GMRES (default): s GMRES steps right-preconditioned
                     by the vertex-star PSC operator; or damped Richardson */
  int sweeps;     /* smoothing steps per level, pre and post (default 5) */
  double tau;     /* Richardson damping (default 2^-d) */
  int transfer;   /* ALS_TRANSFER_ROBUST (default, Eq. (Ptilde)) or ALS_TRANSFER_STANDARD */
  int schur;      /* ALS_SCHUR_P1 (default): S^-1 ~ M_p(1/mu)^-1 + gamma M_p^-1 with the
                     augmentation weight W = M_p; ALS_SCHUR_P2: S^-1 ~ (1+gamma) M_p(1/mu)^-1
                     with W = M_p(1/mu) in A_gamma too (Eq. (P1P2)) */
  int mode;       /* ALS_MODE_FP64 or ALS_MODE_MIXED (FP32 V-cycle, FP64 outer loop) */
  double rtol;    /* FGMRES relative residual reduction (default 1e-8) */
  int maxit;      /* FGMRES iterations, no restart (default 300) */
  int cycle;      /* ALS_CYCLE_V (default) or ALS_CYCLE_F: the coarse correction on each
                     level is an F-cycle from zero followed by a V-cycle from its result
                     (the textbook F-cycle; the paper runs an F-cycle, Sec. 5.1) */
  int fact;       /* block factorisation of Eq. (precond): ALS_FACT_FULL (default, L D U,
                     two cycles per iteration); ALS_FACT_UPPER [[A, B^T], [0, -S]]^-1,
                     ALS_FACT_LOWER [[A, 0], [B, -S]]^-1, ALS_FACT_DIAG diag(A^-1, -S^-1):
                     one cycle per iteration */
  int setup;      /* arithmetic of the patch and coarse inverses: ALS_SETUP_AUTO (default) =
                     FP64 in ALS_MODE_FP64 and double-float (FP32 pairs, about 48 bits) in
                     ALS_MODE_MIXED; ALS_SETUP_FP64 = FP64 in both modes (the mixed cycle then
                     runs on the FP32 roundings of FP64-computed inverses) */
  int order;      /* polynomial order of the velocity: 2 (default, [Q2]^d x P1disc) or 3
                     ([Q3]^d x P2disc, the element of the paper's sinker runs, Table linear,
                     and of its higher-order study, Sec. 5.2.2, Table k; scalar viscosity;
                     nodes 3n+1 per direction; 4^d Gauss points per cell (point data
                     [cell][16] in 2D, [cell][64] in 3D, points x-fastest); pressure per cell
                     the coefficients of the monomials of degree <= 2 in reference
                     coordinates, by degree, x before y before z: {1, xi, eta, xi^2, xi eta,
                     eta^2} in 2D, {1, xi, eta, zeta, xi^2, xi eta, xi zeta, eta^2, eta zeta,
                     zeta^2} in 3D; vertex stars of 5^d nodes (50 / 375 dofs) assembled in
                     FP64 and inverted in FP64, except 3D stars under the setup option's
                     double-float arithmetic (ALS_MODE_MIXED with ALS_SETUP_AUTO); 3D stars
                     take 564 KB (FP64) + 282 KB (FP32) per vertex and about 57 M
                     multiply-adds each to set up) */
  int store;      /* storage of the star inverses the FP32 cycle streams: ALS_STORE_FP32
                     (default), or ALS_STORE_BF16: the block-packed stars (every star, or the
                     interior ones on levels stored split) rounded to bfloat16 to nearest,
                     widened to FP32 on load, every product and sum in FP32 (the optional
                     reduced-precision variant of the scope); boundary stars of split levels,
                     the FP64 cycle and the setup are unchanged.  It halves the smoother's
                     bytes but keeps about 3 significant digits of each inverse, so it is
                     an opt-in for mild problems: with the P2 pairing the FGMRES counts held
                     at DR 1e4 (2D and 3D) and, in 2D, up to DR 1e8 at gamma 1e3 (+3), but
                     the 3D 32^3 solve at DR 1e8, gamma 1e4 did not converge; with P1 it
                     costs a few iterations at DR 1e4 and does not converge from DR 1e6.
                     Order 2, and order 3 in 3D (its wrapped FP32 rows rounded the same way;
                     the interior solves of the FP32 transfers read them too); refused for
                     order 3 in 2D (ALS_EINVAL). */
} als_options;

typedef struct {
  int iterations;     /* FGMRES iterations */
  int vcycles;        /* multigrid cycles applied (2 per iteration with ALS_FACT_FULL, else 1) */
  int converged;
  double res0;        /* ||b||_2 of the augmented, lifted system */
  double res_final;   /* FGMRES residual estimate at exit */
  double solve_ms;    /* wall time of the solve on the context stream */
} als_solve_info;

/* Fills *opt with the defaults listed above. */
void als_default_options(als_options* opt);

/* Setup (Secs. 4-5): copies the coefficients, assembles and inverts the
 * vertex-star patch matrices of levels 1..L-1 (stored as FP64 and FP32
 * inverses), inverts the coarsest A_gamma (dense inverse, kept in FP64) and
 * forms the per-cell Schur-complement blocks of the finest level.  Both
 * inversions use the symmetric sweep; they run in FP64 in ALS_MODE_FP64 and in
 * double-float arithmetic (FP32 pairs, about 48 significant bits) in
 * ALS_MODE_MIXED unless options.setup = ALS_SETUP_FP64; the mixed cycle uses the
 * FP32 inverses.
 * levels = 1: no multigrid; the (1,1) block of the preconditioner is then solved
 * exactly by the dense inverse of A_gamma on the mesh (the exact-A study of Sec. 3,
 * Table exacttopleft); the dense inverse takes (d prod(2n-1))^2 doubles.
 * Mixed mode with the P1 pairing (W = M_p) returns ALS_EINVAL when
 * 2^-24 gamma / mu_min > 0.1 (mu_min: the smallest viscosity, or mu_eff, of all
 * levels' points): the FP32 cycle does not converge there; the P2 pairing has no such
 * limit.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Size limits (ALS_EINVAL): d (k n+1)^d velocity values, d (k+1)^d n^d per-cell
 * outputs and d (2k-1)^d (n+1)^d vertex-star patch outputs (k = options.order;
 * products over the axes) must each stay below 2^31 (the kernels index them with
 * 32 bits). */
als_status als_create(const als_mesh* mesh, const als_coeff* coeff, double gamma, const als_options* opt,
                      void* stream, als_ctx** out);

/* Waits for the context's stream, then frees everything the context owns (device
 * buffers, captured graphs, events, its stream).  NULL: ALS_EINVAL. */
als_status als_destroy(als_ctx* ctx);

/* y = A_gamma x on `level` (Eq. (augstokessys); W = M_p, or M_p(1/mu) with
 * ALS_SCHUR_P2), matrix-free.
 * x, y: device vectors of length d*N_level in precision `prec`
 * (ALS_PREC_FP64: double, ALS_PREC_FP32: float).  Boundary rows: y_D = x_D. */
als_status als_apply_agamma(als_ctx* ctx, int level, int prec, const void* x, void* y);

/* x = one V-cycle (Sec. 4, Fig. algo-outline) for A_gamma x = b on the finest level
 * from x = 0 (pre-smoothing, robust restriction, recursion, coarse Cholesky solve,
 * robust prolongation, post-smoothing).  b, x: device, precision `prec`;
 * ALS_PREC_FP32 runs the whole cycle in FP32 except the FP64 coarse solve. */
als_status als_vcycle(als_ctx* ctx, int prec, const void* b, void* x);

/* Stage entry points (one step of the V-cycle each, device vectors):
 *   als_star_smooth : z = sum_v I_v A_v^-1 I_v^T r on `level` >= 1 (Sec. 4.1)
 *   als_prolong     : xf = P~ xc from level-1 to `level` (Eq. (Ptilde)),
 *                     or P_H xc when the context uses ALS_TRANSFER_STANDARD
 *   als_restrict    : rc = P~^T rf from `level` to level-1
 *   als_coarse_solve: x = A_0^-1 b on the free dofs of level 0 */
als_status als_star_smooth(als_ctx* ctx, int level, int prec, const void* r, void* z);
als_status als_prolong(als_ctx* ctx, int level, int prec, const void* xc, void* xf);
als_status als_restrict(als_ctx* ctx, int level, int prec, const void* rf, void* rc);
als_status als_coarse_solve(als_ctx* ctx, int prec, const void* b, void* x);

/* FP64 system operator of Eq. (augstokessys) on the finest level:
 * [yu; yp] = [[A_gamma, B^T], [B, 0]] [u; p] (device vectors). */
als_status als_apply_stokes(als_ctx* ctx, const double* u, const double* p, double* yu, double* yp);

/* Copies the FP64 inverse of the patch matrix A_v (Sec. 4.1, Eq. (viim)) of
 * vertex `vertex` on `level` as a full m x m row-major matrix to `out` (host or
 * device), m = d*3^d at order 2 and d*5^d at order 3.
 * In ALS_MODE_MIXED the order-2 patches are assembled and inverted in double-float
 * arithmetic (about 48 significant bits) unless options.setup = ALS_SETUP_FP64,
 * else (and at order 3) in FP64.
 * Patch dof order: component-major, node offsets (-1,0,1)^d (order 3: -2..2)
 * x-fastest; rows of nodes outside the domain or on the boundary are identity rows. */
als_status als_patch_inverse(als_ctx* ctx, int level, long long vertex, double* out);

/* Solve the augmented Stokes system (Eqs. (stokessys), (augstokessys)) on the
 * finest level with FGMRES preconditioned by the block factorisation of
 * Eq. (precond) chosen by options.fact: the multigrid cycle of options.cycle for
 * A_gamma, and the Schur approximation of options.schur (P1 or P2, Eq. (P1P2)).
 *   f_qp : [cell][3^d][d] body force at the Gauss points (required)
 *   u_bc : [d][N] nodal Dirichlet values, only boundary entries are read (NULL = 0)
 *   r2   : [cell][d+1] divergence right-hand side (NULL = 0)
 *   u    : [d][N] output velocity including the boundary values
 *   p    : [cell][d+1] output pressure, zero mean
 * Returns ALS_ENOTCONV if rtol was not reached (u, p hold the last iterate). */
als_status als_solve(als_ctx* ctx, const double* f_qp, const double* u_bc, const double* r2, double* u,
                     double* p, als_solve_info* info);

/* ---- Newton's method for the viscoplastic rheology (Sec. 5.3.1) -------------
 * Solves -div(2 mu(eps_II(u)) eps(u)) + grad p = f, -div u = 0 with u = u_D on the
 * boundary, mu(eps_II) = mu_ref tau_y / (2 mu_ref eps_II + tau_y), eps_II = sqrt(eps:eps/2).
 * Starting from u = u_D on the boundary (0 inside) and p = 0, each step linearises at the
 * iterate (the fourth-order coefficient 2 mu [I - (eps (x) T)_sym / (2 eps_II max(tau_y,
 * T_II))], T = 2 mu eps, and mu, evaluated at every level's Gauss points from the finest
 * velocity: rediscretisation, Sec. 5.1), re-runs the setup with it, solves the linearised
 * AL-augmented system for the step with the context's FGMRES to an absolute tolerance of
 * 1e-12 |R_0| (relative at most 1e-2), and backtracks by halving until the residual norm
 * |(R_u, R_p)| falls by a factor (1 - 1e-4 alpha) (after max_halvings failed tries the
 * last halved step is taken).  Stops when |R| <= rtol |R_0|.
 * The context must have tensor coefficients (ALS_COEFF_TENSOR; its initial ones are
 * replaced) and options.schur = ALS_SCHUR_P2 (W = M_p(1/mu), Sec. 5.3.2); either mode.
 *   f_qp : [cell][3^d][d] body force at the finest Gauss points; u_bc : [d][N] nodal
 *          Dirichlet data (boundary entries read; NULL = 0); u, p : outputs (host or device)
 * Returns ALS_ENOTCONV if rtol was not reached within maxit steps (u, p: last iterate). */
typedef struct {
  double mu_ref;      /* reference viscosity (default 1) */
  double tau_y;       /* yield stress (default 1) */
  double rtol;        /* nonlinear residual reduction (default 1e-10) */
  int maxit;          /* Newton steps (default 30) */
  int max_halvings;   /* backtracking halvings per step (default 12) */
} als_newton_params;
typedef struct {
  int iterations;         /* Newton steps taken */
  int linear_iterations;  /* FGMRES iterations over all steps */
  int converged;
  double res0;            /* |(R_u, R_p)| at the initial iterate */
  double res_final;       /* at the last iterate */
} als_newton_info;
void als_newton_default_params(als_newton_params* prm);
als_status als_newton_solve(als_ctx* ctx, const als_newton_params* prm, const double* f_qp, const double* u_bc,
                            double* u, double* p, als_newton_info* info);
/* Residual norm after each step of the last Newton solve (res[0] at the initial iterate)
 * and the FGMRES iterations of each step (linear_its[0] = 0); copies min(cap, count). */
als_status als_newton_history(const als_ctx* ctx, double* res, int* linear_its, int cap, int* count);

/* Re-runs the setup of als_create (patch factorisations, coarse Cholesky,
 * Schur blocks) for new coefficients of the same kind and sizes, reusing every
 * allocation and the captured V-cycle graphs: the per-linearisation setup of
 * a nonlinear (Newton) iteration, Sec. 5.3.  Host or device pointers.
 * The mixed-mode range check of als_create applies; when it refuses, the context
 * holds the new coefficients but stale inverses: call again with valid ones. */
als_status als_update_coefficients(als_ctx* ctx, const als_coeff* coeff);

/* Live timing of the finest-level vertex-star patch kernel inside V-cycles:
 * als_profile(ctx, 1) makes subsequent V-cycles record a CUDA event pair around
 * each such launch on the stream it runs on.  With graph replay (the default) the
 * cycle is captured a second time with event-record nodes and that graph is
 * replayed for one cycle in every 8 (the first after als_profile and every 8th
 * after it); the other cycles replay the plain graph, so timing barely slows the
 * run it measures.  Without graphs (ALS_NO_GRAPH=1) every cycle is timed.
 * als_profile_read() returns the summed kernel time in ms and the number of
 * launches measured since the previous read, and restarts the accumulation.
 * als_profile(ctx, 0) turns it off. */
als_status als_profile(als_ctx* ctx, int on);
als_status als_profile_read(als_ctx* ctx, double* total_ms, long long* launches);
/* As als_profile_read for one kernel class: kind 0 = the finest-level star-patch
 * kernel (same as als_profile_read), kind 1 = the finest-level operator-apply cell
 * kernel of the GMRES smoother steps (its node gather excluded).  Each kind
 * accumulates separately and is reset by its own read.  ALS_EINVAL for another kind. */
als_status als_profile_read_kernel(als_ctx* ctx, int kind, double* total_ms, long long* launches);

/* Factor injection (tests and inspection): replace the setup's inverses by the
 * caller's, so that the cycle can be compared with another implementation on
 * identical factors (Sec. 4.1 patches, Sec. 5.1 coarse solve).
 *   als_load_patch_inverses: `packed` (host or device) holds, for every vertex of
 *     `level` (1 <= level < levels, vertex index x-fastest), the FP64 inverse of its
 *     patch matrix in the layout of als_star_smooth_static's `inv` (upper triangle by
 *     diagonals, padded to a multiple of 4 entries; identity rows at absent and
 *     boundary nodes): np = d (2k - 1)^d dofs a patch at order k (18 / 81 at k = 2,
 *     50 / 375 at k = 3), (n_l + 1)^d blocks of round_up(np (np + 1) / 2, 4) doubles;
 *     the FP32 copies of the cycle are rounded from it.
 *   als_load_coarse_inverse: `inv` (host or device) is the nfree x nfree row-major
 *     inverse of the coarsest A_gamma on its free dofs, nfree = d prod(k n_0 - 1),
 *     free dofs ordered component-major, then interior nodes x-fastest.
 * Both copy synchronously and read exactly those sizes from the caller's buffer (the
 * Python binding checks the length and dtype first); als_update_coefficients
 * overwrites them again. */
als_status als_load_patch_inverses(als_ctx* ctx, int level, const double* packed);
als_status als_load_coarse_inverse(als_ctx* ctx, const double* inv);

/* Test switch: poll limit of the FP32 star-smoother kernel's wait for its inverse
 * blocks (polls < 0 restores the default, about a second of polling).  With 0 the
 * first wait of every CTA gives up at once: the call that ran the smoother then
 * returns ALS_ETIMEOUT (after the kernel has waited, at the default limit, for the
 * copies it had issued), and the next call with the default limit works normally.
 * Drops the captured cycles (they embed the limit). */
als_status als_set_wait_limit(als_ctx* ctx, int polls);

/* Residual history of the context's last solve: out[0] = |b| of the augmented,
 * lifted system, out[k] = the FGMRES residual estimate after iteration k.  Copies
 * min(cap, count) values; *count gets the length (iterations + 1). */
als_status als_solve_history(const als_ctx* ctx, double* out, int cap, int* count);

/* Process-wide number of kernels this library has launched (a replay of a
 * captured V-cycle counts its kernel nodes). */
long long als_kernel_launches(void);

/* Allocation-free star smoother.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they
 * smooth -- real-time loops that reserve all device memory up front, plugins
 * whose host framework owns the allocator, or code where the implicit device
 * synchronisation of an allocation is not acceptable.  It computes the same z as
 * als_star_smooth, but without a context: the caller passes the mesh, the packed
 * patch inverses, r and z (all device memory it already owns), and the per-patch
 * scratch the smoother needs between its two kernels is a fixed device array of
 * ALS_STATIC_SCRATCH_BYTES inside this library, which every GPU that loads the
 * library holds until the process exits.
 *   dim, n : mesh of the level (n[k] cells per direction, n[2] ignored in 2D)
 *   prec   : ALS_PREC_FP64 (double inv/r/z) or ALS_PREC_FP32 (float)
 *   inv    : device, one block per vertex (vertex index x-fastest), each block
 *            the upper triangle of the (d*3^d)^2 inverse stored by diagonals,
 *            entries (i, i+t) for t = 0.., i = 0..np-1-t, padded to a multiple
 *            of 4 entries; patch dof order as in als_patch_inverse
 *   r, z   : device velocity vectors of the level (boundary entries of z = 0)
 *   stream : cudaStream_t the two kernels are queued on; the call returns
 *            without waiting for them
 * Returns ALS_EINVAL for n[k] outside [1, 4096] or when
 * (n+1)^d * d*3^d * sizeof(element) exceeds ALS_STATIC_SCRATCH_BYTES (32 MiB: e.g.
 * up to 32^3 hexes in FP64, 45^3 in FP32), and ALS_ECUDA when a launch fails.
 * The first call on a device (with that device current) looks up the array's
 * device address and the SM count; make that first call before any stream capture.
 * Nothing is allocated and nothing needs to start at zero, but every call
 * shares the one array: calls that overlap on the GPU race. */
#define ALS_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
als_status als_star_smooth_static(int dim, const int* n, int prec, const void* inv, const void* r, void* z,
                                  void* stream);

/* Measured FP32 and FP64 fused multiply-add throughput of the current GPU's
 * CUDA cores, in TFLOP/s (2 flops per FMA), for the ALU rooflines.  Runs two
 * short kernels (about 0.1 s) on `stream` (a cudaStream_t) and waits for them;
 * allocates and frees 2 KiB of device memory.  Returns ALS_EINVAL for NULL
 * outputs, ALS_ENOMEM or ALS_ECUDA on a runtime failure. */
als_status als_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, void* stream);

/* ---- Batches of independent instances (serving-style sweeps) ----------------
 * A batch holds `count` independent problems, each with its own mesh, level
 * count, coefficients, gamma and options (2D and 3D may be mixed); instance i
 * is a full context (als_batch_context gives it for the per-instance calls).
 * als_batch_solve runs all solves together: each round queues one FGMRES
 * iteration of every unfinished instance (the instances' own FGMRES kernels on
 * their own streams, the preconditioner's cycles in the batch's cycle form, see
 * ALS_BATCH_MERGED), then waits once; results are bitwise those of als_solve on
 * the same instance.  als_batch_vcycle applies one multigrid cycle to every
 * instance in the batch's cycle form (FP64 cycles: always the graph of the
 * instances' captured cycles).
 * Arrays are indexed by instance: meshes/coeffs/gammas[count]; opts[count] or
 * NULL (defaults); f_qp, u_bc, r2, u, p, b, x: arrays of count pointers with
 * the meaning and layout of the single-instance calls (u_bc, r2 may be NULL
 * arrays or hold NULL entries); infos[count] or NULL.
 * Errors: als_batch_create returns the first failing instance's status (and
 * creates nothing); als_batch_solve finishes every instance and returns the
 * first non-OK status (the message names the instance); als_batch_vcycle needs
 * graph capture on and profiling off in every instance (ALS_EINVAL otherwise). */
typedef struct als_batch als_batch;
als_status als_batch_create(int count, const als_mesh* meshes, const als_coeff* coeffs, const double* gammas,
                            const als_options* opts, void* stream, als_batch** out);
als_status als_batch_destroy(als_batch* batch);
als_status als_batch_context(als_batch* batch, int i, als_ctx** ctx);
als_status als_batch_solve(als_batch* batch, const double* const* f_qp, const double* const* u_bc,
                           const double* const* r2, double* const* u, double* const* p, als_solve_info* infos);
als_status als_batch_vcycle(als_batch* batch, int prec, const void* const* b, void* const* x);
const char* als_batch_last_error(const als_batch* batch);

/* Execution form of a batch's FP32 multigrid cycles (those of als_batch_vcycle with
 * prec FP32, and the preconditioner cycles of a mixed-mode als_batch_solve):
 *   ALS_BATCH_MERGED    one launch per level operation for each group of instances:
 *                       every operator apply, star-product sweep, transfer, GMRES step
 *                       and the coarse solve of the group's V-cycles runs as one merged
 *                       kernel launch whose grid is the flattened (instance, tile) work
 *                       list; the hierarchies of a group are aligned at their coarsest
 *                       level, each group's merged cycle is captured as a CUDA graph and
 *                       the groups run as independent branches of one graph (see
 *                       als_batch_merged_plan for the grouping and the autotuner); each
 *                       instance's cycle of Sec. 4 is unchanged.
 *   ALS_BATCH_BRANCHES  one graph launch whose independent branches are the
 *                       instances' own captured cycles (solves: one stream each).
 * Every instance's results are bitwise those of its single-instance calls in both
 * forms.  MERGED needs, in every instance: order 2, scalar viscosity, the GMRES
 * smoother with at most 8 steps, the V-cycle, kernel timing off, and the sweeps and
 * transfer of instance 0; a mixed-mode solve also needs the full block factorisation
 * (ALS_FACT_FULL), else the solve runs in the BRANCHES form.  A merged solve joins
 * each group's cycles with its instances' own streams by events, so a batch wants
 * more hardware work queues than the default 8 (CUDA_DEVICE_MAX_CONNECTIONS=32 in
 * the environment before CUDA starts).  als_batch_create picks MERGED when every
 * instance qualifies.  als_batch_set_mode returns ALS_EINVAL for an unknown mode or,
 * for MERGED, when an instance does not qualify (the message says which and why).
 * als_batch_get_mode reads the mode. */
enum { ALS_BATCH_MERGED = 0, ALS_BATCH_BRANCHES = 1 };
als_status als_batch_set_mode(als_batch* batch, int mode);
als_status als_batch_get_mode(const als_batch* batch, int* mode);

/* Plan of the merged cycles (made on the first merged FP32 cycle or mixed solve):
 * the instances are split into groups, each group's cycles merged into one launch
 * per level operation, and the groups' captured cycles run as independent branches
 * of one graph, so that one group's latency-bound coarse levels overlap another's
 * bandwidth-bound fine levels.  The autotuner builds and times (three cycles, CUDA
 * events) each grouping that gives a distinct partition -- 0: one group, 1: by
 * dimension, 2: by dimension and level count, 3: by shape (dimension, cells, levels),
 * 4: by shape in chunks of at most four instances -- and keeps the fastest; within a
 * group it times the three star-kernel variants of every merged star-product and
 * interior-solve launch (0: TMA ring, 2 stages; 1: 3 stages; 2: direct loads).
 * als_batch_merged_plan: the chosen grouping, the number of groups, ms[5] (optional)
 * the measured time per cycle of each grouping (-1: not built, same partition as an
 * earlier one), *kernels (optional) the kernel launches of one merged cycle of the
 * whole batch.  als_batch_merged_tune: for group `group` and level index `level`
 * (0 = coarsest, 1 <= level < the group's largest level count), the variants chosen
 * for the merged star products and interior solves, ms[6] (optional) the time per
 * launch of each variant (products, then interior solves), and instances (optional,
 * room for count entries) the batch indices of the group's instances in order.
 * ALS_EINVAL: NULL batch or required output, index out of range, or no plan yet. */
als_status als_batch_merged_plan(const als_batch* batch, int* grouping, int* groups, float* ms, long long* kernels);
/* Fixes the grouping of the merged cycles (0 .. 4 as above) or, with -1, lets the
 * tuner choose again; drops the current plan (made again on the next merged call).
 * ALS_EINVAL for a NULL batch or a grouping out of range. */
als_status als_batch_set_grouping(als_batch* batch, int grouping);
als_status als_batch_merged_tune(const als_batch* batch, int group, int level, int* products_variant,
                                 int* interior_variant, float* ms, int* instances);

/* Autotuner record of a smoothed level (1 <= level < levels).  Before the FP32
 * cycle is first captured, each level times its FP32 star-patch kernel variants
 * (0: TMA ring with 2 stages, 1: TMA ring with 3 stages, 2: direct 16-byte loads;
 * one warm-up and three timed launches each) and keeps the fastest.  *variant gets
 * the choice (-1 before tuning); ms[3] (optional) the measured time per launch of
 * each variant.  ALS_PATCH_KERNEL = tma2 | tma3 | direct in the environment forces
 * a variant. */
als_status als_autotune_info(als_ctx* ctx, int level, int* variant, float* ms);
/* Sets the FP32 patch-kernel variant of a level (0, 1, 2 as above; -1 = tune again
 * before the next capture); the captured cycles are dropped and recaptured. */
als_status als_set_patch_kernel(als_ctx* ctx, int level, int variant);

/* Last error message of the context (never NULL; "" when none).  With ctx NULL:
 * the message of the calling thread's last failed als_create or als_batch_create
 * ("" when its last call succeeded). */
const char* als_last_error(const als_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ALSTOKES_H */
