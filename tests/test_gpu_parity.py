"""GPU parity: every C-ABI entry point against the FP64 oracle on the same seeded inputs.

Tolerances (relative l2):
  * FP64 operator applies, transfers, coarse solve: 1e-12 (the FP64 parity bar);
  * FP64 patch inverses / smoother / V-cycle: the oracle factors each patch with
    LAPACK and the GPU with its own Cholesky, so the two inverses differ by
    O(cond(A_v) eps); the tests use well-conditioned cases at 1e-12 and a
    cond-scaled bound for the extreme-contrast cases;
  * FP32 paths: 2e-5 (single-precision rounding of O(100)-term sums).
"""
import numpy as np
import pytest

from gpu_helpers import context, dev, host, oracle, random_free, rel, sinker, torch  # noqa: F401
from oracle.fem import Level
from oracle.mg import star_dofs, all_vertices
from oracle.stokes import StokesSolver

pytestmark = pytest.mark.gpu

from paper_2107_00820_gb300 import alstokes as A  # noqa: E402


# --------------------------------------------------------------------------
# a1: A_gamma apply
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,n,levels", [(2, 8, 2), (2, (12, 6), 2), (3, 4, 2), (3, 6, 1)])
@pytest.mark.parametrize("gamma", [0.0, 1e4])
def test_apply_agamma_fp64(d, n, levels, gamma):
    pb = sinker(d, n, levels, gamma, dr=1e6, seed=1)
    ctx = context(pb)
    H = oracle(pb, smoother="richardson", steps=1)
    for lvl in range(levels):
        lv = H.levels[lvl]
        x = np.random.default_rng(lvl).standard_normal(lv.mesh.nu)   # boundary entries nonzero too
        y = torch.zeros(lv.mesh.nu, dtype=torch.float64, device="cuda")
        ctx.apply_agamma(dev(x), y, lvl)
        assert rel(host(y), lv.A @ x) <= 1e-12


@pytest.mark.parametrize("d,n", [(2, 16), (3, 6)])
def test_apply_agamma_fp32(d, n):
    pb = sinker(d, n, 1, 1e3, dr=1e4, seed=2)
    ctx = context(pb)
    lv = Level(d, pb.n, pb.mu[0], pb.gamma)
    x = np.random.default_rng(3).standard_normal(lv.mesh.nu)
    y = torch.zeros(lv.mesh.nu, dtype=torch.float32, device="cuda")
    ctx.apply_agamma(dev(x, torch.float32), y, 0, A.ALS_PREC_FP32)
    assert rel(host(y), lv.A @ x.astype(np.float32).astype(np.float64)) <= 2e-5


@pytest.mark.parametrize("d", [2, 3])
def test_apply_agamma_tensor_fp64(d):
    """a2: anisotropic 4th-order tensor C at every point (Eq. (stokes-lin))."""
    n = 4 if d == 3 else 8
    rng = np.random.default_rng(7)
    nm = 3 if d == 2 else 6
    ncells, nq = n ** d, 3 ** d
    M = rng.standard_normal((ncells, nq, nm, nm))
    C = np.einsum("cqij,cqkj->cqik", M, M) + 0.5 * np.eye(nm)
    iu = np.triu_indices(nm)
    Cp = np.ascontiguousarray(C[:, :, iu[0], iu[1]])
    mu_eff = np.ascontiguousarray(C[:, :, 0, 0] / 2)
    from paper_2107_00820_gb300 import Context
    ctx = Context(d, n, 1, [Cp], 10.0, mu_eff=[mu_eff])
    lv = Level(d, n, Cp, 10.0, kind="tensor", mu_eff=mu_eff)
    x = rng.standard_normal(lv.mesh.nu)
    y = torch.zeros_like(dev(x))
    ctx.apply_agamma(dev(x), y, 0)
    assert rel(host(y), lv.A @ x) <= 1e-12


@pytest.mark.parametrize("d,n", [(2, 8), (3, 5)])
def test_apply_agamma_tensor_fp32(d, n):
    """a2 in FP32 (the mixed cycle's operator): the 3D cell kernel stages each cell's
    27 x 21 coefficients in shared memory; element-wise against the oracle on the same
    FP32-rounded input, at FP32 rounding."""
    rng = np.random.default_rng(17)
    nm = 3 if d == 2 else 6
    ncells, nq = n ** d, 3 ** d
    M = rng.standard_normal((ncells, nq, nm, nm))
    C = np.einsum("cqij,cqkj->cqik", M, M) + 0.5 * np.eye(nm)
    iu = np.triu_indices(nm)
    Cp = np.ascontiguousarray(C[:, :, iu[0], iu[1]])
    mu_eff = np.ascontiguousarray(C[:, :, 0, 0] / 2)
    from paper_2107_00820_gb300 import Context
    ctx = Context(d, n, 1, [Cp], 10.0, mu_eff=[mu_eff])
    lv = Level(d, n, Cp, 10.0, kind="tensor", mu_eff=mu_eff)
    x = rng.standard_normal(lv.mesh.nu)
    y = torch.zeros(lv.mesh.nu, dtype=torch.float32, device="cuda")
    ctx.apply_agamma(dev(x, torch.float32), y, 0, A.ALS_PREC_FP32)
    ref = lv.A @ x.astype(np.float32).astype(np.float64)
    assert rel(host(y), ref) <= 2e-5


@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
def test_apply_stokes_fp64(d, n):
    pb = sinker(d, n, 2, 1e2, dr=1e4, seed=4)
    ctx = context(pb)
    s = StokesSolver(oracle(pb, smoother="richardson", steps=1))
    rng = np.random.default_rng(5)
    u = rng.standard_normal(s.nu)
    p = rng.standard_normal(s.np_)
    yu = torch.zeros(s.nu, dtype=torch.float64, device="cuda")
    yp = torch.zeros(s.np_, dtype=torch.float64, device="cuda")
    ctx.apply_stokes(dev(u), dev(p), yu, yp)
    ref = s.matvec(np.concatenate([u, p]))
    assert rel(host(yu), ref[: s.nu]) <= 1e-12
    assert rel(host(yp), ref[s.nu:]) <= 1e-12


# --------------------------------------------------------------------------
# a3/a4: patch setup and the star smoother
# --------------------------------------------------------------------------
def _patch_cond(H, lvl, v):
    lv = H.levels[lvl]
    idx = star_dofs(lv.mesh, v)
    Av = lv.A[idx][:, idx].toarray()
    return np.linalg.cond(Av), idx, Av


@pytest.mark.parametrize("d,n,gamma,dr", [(2, 8, 1.0, 1e2), (2, 8, 1e4, 1e6), (3, 4, 1e2, 1e4)])
def test_patch_inverses_sampled(d, n, gamma, dr):
    pb = sinker(d, n, 2, gamma, dr, seed=6)
    ctx = context(pb)
    H = oracle(pb, smoother="richardson", steps=1)
    m = H.levels[1].mesh
    verts = all_vertices(m)
    rng = np.random.default_rng(0)
    picks = list(rng.choice(len(verts), size=min(12, len(verts)), replace=False)) + [0, len(verts) - 1]
    NB = 3 ** d
    for vid in picks:
        v = verts[vid]
        cond, idx, Av = _patch_cond(H, 1, v)
        full = ctx.patch_inverse(1, int(vid))
        # rows of the GPU patch that correspond to free nodes, in oracle order
        keep = []
        for a in range(d):
            for o in range(NB):
                g = 2 * v + (np.array([o % 3, (o // 3) % 3, o // 9][:d]) - 1)
                if np.all(g > 0) and np.all(g < np.array(m.nn) - 1):
                    keep.append(a * NB + o)
        keep = np.array(keep)
        assert len(keep) == len(idx)
        got = full[np.ix_(keep, keep)]
        ref = np.linalg.inv(Av)
        tol = max(1e-12, 20 * cond * 2.2e-16)
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (vid, cond)
        # identity rows for absent nodes
        other = np.setdiff1d(np.arange(d * NB), keep)
        if len(other):
            assert np.allclose(full[np.ix_(other, other)], np.eye(len(other)))


@pytest.mark.parametrize("d,n", [(2, 16), (3, 4)])
@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_star_smoother(d, n, prec):
    pb = sinker(d, n, 2, 1e2, dr=1e3, seed=8)
    ctx = context(pb)
    H = oracle(pb, smoother="richardson", steps=1)
    lv = H.levels[1]
    r = random_free(lv, 9)
    dt = torch.float64 if prec == A.ALS_PREC_FP64 else torch.float32
    z = torch.zeros(lv.mesh.nu, dtype=dt, device="cuda")
    ctx.star_smooth(1, dev(r, dt), z, prec)
    ref = H.patches[1].apply(r)
    assert rel(host(z), ref) <= (1e-11 if prec == A.ALS_PREC_FP64 else 1e-4)


# --------------------------------------------------------------------------
# a5/a6: robust prolongation and restriction, standard transfers
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
@pytest.mark.parametrize("transfer", [A.ALS_TRANSFER_ROBUST, A.ALS_TRANSFER_STANDARD])
def test_transfers_fp64(d, n, transfer):
    pb = sinker(d, n, 2, 1e2, dr=1e3, seed=10)
    ctx = context(pb, transfer=transfer)
    H = oracle(pb, smoother="richardson", steps=1, transfer="robust" if transfer == 0 else "standard")
    c, f = H.levels[0], H.levels[1]
    xc = random_free(c, 11)
    xf = torch.zeros(f.mesh.nu, dtype=torch.float64, device="cuda")
    ctx.prolong(1, dev(xc), xf)
    assert rel(host(xf), H.P[1] @ xc) <= 1e-11
    rf = random_free(f, 12)
    rc = torch.zeros(c.mesh.nu, dtype=torch.float64, device="cuda")
    ctx.restrict(1, dev(rf), rc)
    assert rel(host(rc), H.P[1].T @ rf) <= 1e-11


# --------------------------------------------------------------------------
# a7: coarse solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,n", [(2, 4), (2, 8), (3, 2), (3, 4)])
def test_coarse_solve(d, n):
    pb = sinker(d, n, 1, 1e2, dr=1e4, seed=13)
    ctx = context(pb)
    H = oracle(pb, smoother="richardson", steps=1)
    b = random_free(H.levels[0], 14)
    x = torch.zeros_like(dev(b))
    ctx.coarse_solve(dev(b), x)
    ref = H.coarse_solve(b)
    cond = np.linalg.cond(H.levels[0].A.toarray())
    assert rel(host(x), ref) <= max(1e-12, 10 * cond * 2.2e-16)


# --------------------------------------------------------------------------
# a8: V-cycle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("smoother", [A.ALS_SMOOTH_RICHARDSON, A.ALS_SMOOTH_GMRES])
@pytest.mark.parametrize("d,n,levels", [(2, 16, 3), (3, 8, 3)])
def test_vcycle_fp64(smoother, d, n, levels):
    pb = sinker(d, n, levels, 1.0, dr=1e2, seed=15)
    ctx = context(pb, smoother=smoother, sweeps=2)
    H = oracle(pb, smoother="gmres" if smoother == A.ALS_SMOOTH_GMRES else "richardson", steps=2)
    b = random_free(H.levels[-1], 16)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.vcycle(b)) <= 1e-12


@pytest.mark.parametrize("sweeps,transfer", [(1, A.ALS_TRANSFER_ROBUST), (8, A.ALS_TRANSFER_STANDARD),
                                             (10, A.ALS_TRANSFER_ROBUST)])
def test_vcycle_fp64_gmres_steps(sweeps, transfer):
    """GMRES smoothing with 1 and 8 steps (fused kernels, unnormalised basis, residual
    from the Arnoldi relation) and 10 steps (the explicit path), both transfers."""
    pb = sinker(2, 16, 3, 1.0, dr=1e2, seed=16)
    ctx = context(pb, smoother=A.ALS_SMOOTH_GMRES, sweeps=sweeps, transfer=transfer)
    H = oracle(pb, smoother="gmres", steps=sweeps,
               transfer="robust" if transfer == A.ALS_TRANSFER_ROBUST else "standard")
    b = random_free(H.levels[-1], 17)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.vcycle(b)) <= 1e-12


@pytest.mark.parametrize("smoother", [A.ALS_SMOOTH_RICHARDSON, A.ALS_SMOOTH_GMRES])
@pytest.mark.parametrize("d,n,levels", [(2, 16, 4), (3, 8, 3)])
def test_fcycle_fp64(smoother, d, n, levels):
    """F-cycle (F-cycle then V-cycle from its result on each coarser level)."""
    pb = sinker(d, n, levels, 1.0, dr=1e2, seed=25)
    ctx = context(pb, smoother=smoother, sweeps=2, cycle=A.ALS_CYCLE_F)
    H = oracle(pb, smoother="gmres" if smoother == A.ALS_SMOOTH_GMRES else "richardson", steps=2, cycle="F")
    b = random_free(H.levels[-1], 26)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.cycle(b)) <= 1e-12
    assert rel(host(x), H.vcycle(b)) > 1e-6          # really a different cycle


def _max_patch_cond(H, lvl, count=40):
    m = H.levels[lvl].mesh
    verts = all_vertices(m)
    picks = np.random.default_rng(0).choice(len(verts), size=min(count, len(verts)), replace=False)
    return max(_patch_cond(H, lvl, verts[i])[0] for i in picks)


def _cycle_cond(H, lvl, count=40):
    """Condition number that scales the FP64 rounding of a cycle: the worst of the
    sampled patch matrices (the smoother's local inverses) and of the coarsest
    operator (the coarse solve's dense inverse); both inverses are computed to
    about cond * eps relative accuracy."""
    lv0 = H.levels[0]
    f = np.flatnonzero(lv0.free)
    c0 = np.linalg.cond(lv0.A.toarray()[np.ix_(f, f)])
    return max(_max_patch_cond(H, lvl, count), c0)


@pytest.mark.parametrize("smoother", [A.ALS_SMOOTH_GMRES, A.ALS_SMOOTH_RICHARDSON])
@pytest.mark.parametrize("d,n,levels", [(2, 32, 4), (3, 8, 3)])
def test_vcycle_extreme_contrast(d, n, levels, smoother):
    """gamma = 1e4, DR = 1e8 (cond(A_v) ~ 1e12).  With its own inverses the FP64 cycle
    differs from the oracle's by the two factorisations' cond * eps; with the oracle's
    inverses injected both cycles apply the same matrices and differ only in the order and
    grouping of their sums.  The cycle itself amplifies rounding there: valid reorderings
    of the oracle's own sums move its output by 1e-9 .. 1e-8, and the probabilistic
    rounding model of tests/rounding_model.py by ~4e-7 (against ~1e-11 at moderate contrast,
    where the 1e-12 bar holds: test_vcycle_fp64), so the bar is 3x that model's spread.
    Both cycles must also reduce the residual equally well."""
    from injection import inject, load_into
    from rounding_model import cycle_rounding_spread
    sm = "gmres" if smoother == A.ALS_SMOOTH_GMRES else "richardson"
    pb = sinker(d, n, levels, 1e4, dr=1e8, seed=17)
    ctx = context(pb, sweeps=3, smoother=smoother)
    H = oracle(pb, steps=3, smoother=sm)
    A_f = H.levels[-1].A
    b = random_free(H.levels[-1], 18)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    ref = H.vcycle(b)
    cond = _cycle_cond(H, levels - 1)
    assert rel(host(x), ref) <= max(1e-10, 100 * cond * 2.2e-16), cond
    r_ref = np.linalg.norm(b - A_f @ ref) / np.linalg.norm(b)
    r_gpu = np.linalg.norm(b - A_f @ host(x)) / np.linalg.norm(b)
    assert abs(r_gpu - r_ref) <= 0.01 * r_ref
    load_into(ctx, H, inject(H))
    ref = H.vcycle(b)
    spread = cycle_rounding_spread(H, b)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    err = rel(host(x), ref)
    assert err <= 3 * spread, (err, spread)


@pytest.mark.parametrize("d,n,levels", [(2, 32, 4), (3, 8, 3)])
def test_vcycle_fp32_within_its_precision_range(d, n, levels):
    """The FP32 cycle evaluates gamma div u and the patch inverses in single
    precision; with W = M_p its relative error grows like eps32 * gamma / mu_min.
    At gamma / mu_min = 1e5 (gamma 10, DR 1e8) it must smooth as well as FP64."""
    pb = sinker(d, n, levels, 10.0, dr=1e8, seed=17)
    ctx = context(pb, sweeps=3)
    H = oracle(pb, steps=3)
    A_f = H.levels[-1].A
    b = random_free(H.levels[-1], 18)
    ref = H.vcycle(b)
    r_ref = np.linalg.norm(b - A_f @ ref) / np.linalg.norm(b)
    x32 = torch.zeros(b.shape[0], dtype=torch.float32, device="cuda")
    ctx.vcycle(dev(b, torch.float32), x32, A.ALS_PREC_FP32)
    r32 = np.linalg.norm(b - A_f @ host(x32)) / np.linalg.norm(b)
    assert r32 <= 1.5 * r_ref + 1e-4, (r32, r_ref)


@pytest.mark.parametrize("d,n,levels", [(2, 32, 3), (3, 8, 3)])
def test_patch_kernel_variants_and_autotuner(d, n, levels):
    """Every FP32 patch-kernel variant (TMA ring with 2 or 3 stages, direct loads)
    gives the FP32 cycle to single-precision accuracy of the FP64 oracle cycle; the
    autotuner picks one of them and records the times it measured."""
    pb = sinker(d, n, levels, 10.0, dr=1e2, seed=41)
    H = oracle(pb, steps=2)
    b = random_free(H.levels[-1], 42)
    ref = H.vcycle(b)
    ctx = context(pb, sweeps=2)
    x32 = torch.zeros(b.shape[0], dtype=torch.float32, device="cuda")
    ctx.vcycle(dev(b, torch.float32), x32, A.ALS_PREC_FP32)
    for lvl in range(1, levels):
        v, ms = ctx.autotune_info(lvl)
        assert v in (0, 1, 2) and all(t > 0 for t in ms) and ms[v] == min(ms), (lvl, v, ms)
    assert rel(host(x32), ref) <= 1e-4
    xs = []
    for variant in (0, 1, 2):
        for lvl in range(1, levels):
            ctx.set_patch_kernel(lvl, variant)
        x = torch.zeros_like(x32)
        ctx.vcycle(dev(b, torch.float32), x, A.ALS_PREC_FP32)
        assert rel(host(x), ref) <= 1e-4, variant
        assert ctx.autotune_info(1)[0] == variant
        xs.append(x)
    # the variants differ in staging and occupancy, not in arithmetic: the same bits
    assert all(torch.equal(xs[0], y) for y in xs[1:])


# --------------------------------------------------------------------------
# a9/a10: full solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,n,levels,gamma,dr", [(2, 16, 3, 1e2, 1e4), (3, 8, 2, 1e3, 1e4)])
def test_solve_fp64_matches_oracle(d, n, levels, gamma, dr):
    pb = sinker(d, n, levels, gamma, dr, seed=19)
    ctx = context(pb, rtol=1e-8)
    s = StokesSolver(oracle(pb))
    uo, po, its, hist = s.solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged == 1
    assert abs(info.iterations - its) <= 0, (info.iterations, its)
    assert rel(u, uo) <= 1e-9 and rel(p, po) <= 1e-8


@pytest.mark.parametrize("fact,name", [(A.ALS_FACT_UPPER, "upper"), (A.ALS_FACT_LOWER, "lower"),
                                       (A.ALS_FACT_DIAG, "diag")])
def test_solve_factorisation_types(fact, name):
    """Block-triangular and block-diagonal forms of Eq. (precond), FP64, F-cycle."""
    pb = sinker(2, 16, 3, 1e2, dr=1e4, seed=27)
    ctx = context(pb, rtol=1e-8, fact=fact, cycle=A.ALS_CYCLE_F)
    s = StokesSolver(oracle(pb, cycle="F"), fact=name)
    uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged == 1 and info.iterations == its, (info.iterations, its)
    assert info.vcycles == its
    assert rel(u, uo) <= 1e-9 and rel(p, po) <= 1e-8


def test_solve_manufactured_config():
    """Smallest configuration: 2D 16x16, mu = 1, gamma = 1e4, 2 levels, 2 sweeps, rtol 1e-10."""
    from synthetic.problems import manufactured_problem
    pb = manufactured_problem(16, 2, 1e4)
    ctx = context(pb, sweeps=2, rtol=1e-10)
    s = StokesSolver(oracle(pb, steps=2))
    uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-10)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its
    assert rel(u, uo) <= 1e-9


def _true_residual(solver, pb, u, p):
    """Relative residual |b - K x| / |b| of (u, p) in the oracle's lifted, augmented system
    (x = (u - u_D, p); the pressure constant is in the kernel of K)."""
    b, uD = solver.rhs(pb.f, pb.u_bc)
    r = b - solver.matvec(np.concatenate([u - uD, p]))
    return float(np.linalg.norm(r) / np.linalg.norm(b))


@pytest.mark.parametrize("d,n,levels", [(2, 32, 4), (3, 8, 2)])
def test_solve_mixed_precision(d, n, levels):
    """The mixed path (FP32 cycle inside FP64 FGMRES) reaches rtol 1e-8 within +2
    iterations of the FP64 path, with a true residual (evaluated by the oracle) that meets
    the tolerance; run on to rtol 1e-11 (the FP64 outer loop refining the FP32 cycle's
    corrections) it lies within 1e-7 of the converged oracle solution in velocity and
    pressure.  (A relative residual of 1e-8 alone leaves a solution error of up to
    cond * 1e-8 in any precision: the oracle's own 1e-8 iterate is 2e-8 (u) / 5e-7 (p) away
    from its solution here.)"""
    pb = sinker(d, n, levels, 1e3, dr=1e6, seed=21)
    ref = context(pb, rtol=1e-8)
    s = StokesSolver(oracle(pb))
    uo, po, _, _ = s.solve(pb.f, pb.u_bc, rtol=1e-12)
    _, _, its8, _ = s.solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = context(pb, rtol=1e-8, mode=A.ALS_MODE_MIXED).solve(pb.f, pb.u_bc)
    _, _, info64 = ref.solve(pb.f, pb.u_bc)
    assert info64.iterations == its8
    assert info.converged and info.iterations <= info64.iterations + 2
    assert _true_residual(s, pb, u, p) <= 1.5e-8
    u, p, info = context(pb, rtol=1e-11, mode=A.ALS_MODE_MIXED).solve(pb.f, pb.u_bc)
    assert info.converged
    assert rel(u, uo) <= 1e-7 and rel(p, po) <= 1e-7, (rel(u, uo), rel(p, po))


def test_solve_device_buffers():
    pb = sinker(2, 16, 3, 1e2, dr=1e4, seed=23)
    ctx = context(pb)
    u_h, p_h, _ = ctx.solve(pb.f, pb.u_bc)
    u = torch.zeros(ctx.nu(), dtype=torch.float64, device="cuda")
    p = torch.zeros(ctx.npres(), dtype=torch.float64, device="cuda")
    ctx.solve(dev(pb.f), dev(pb.u_bc), None, u, p)
    # deterministic accumulation order: host and device buffers give identical bits
    assert np.array_equal(host(u), u_h) and np.array_equal(host(p), p_h)
    u2, p2, _ = ctx.solve(pb.f, pb.u_bc)
    assert np.array_equal(u2, u_h) and np.array_equal(p2, p_h)


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------
def test_invalid_arguments_and_non_spd():
    from paper_2107_00820_gb300 import ALSError, Context
    pb = sinker(2, 8, 2, 1.0, dr=1e2)
    with pytest.raises(ALSError) as e:
        Context(2, 6, 3, pb.mu, 1.0)            # 6 not divisible by 4
    assert e.value.status == A.ALS_EINVAL
    with pytest.raises(ALSError) as e:
        Context(1, 8, 2, pb.mu, 1.0)
    assert e.value.status == A.ALS_EINVAL
    bad = [-m for m in pb.mu]                    # negative viscosity: patch matrices not SPD
    with pytest.raises(ALSError) as e:
        Context(2, 8, 2, bad, 0.0)
    assert e.value.status == A.ALS_ENOTSPD
    ctx = context(pb)
    with pytest.raises(ALSError):
        ctx.apply_agamma(torch.zeros(ctx.nu(), dtype=torch.float64, device="cuda"),
                         torch.zeros(ctx.nu(), dtype=torch.float64, device="cuda"), level=7)


# --------------------------------------------------------------------------
# a2 through the whole hierarchy: anisotropic tensor viscosity (Eq. (stokes-lin))
# --------------------------------------------------------------------------
def _tensor_problem(d, n, levels, gamma, seed=1):
    from synthetic.problems import viscoplastic_problem
    return viscoplastic_problem(d, n, levels, gamma=gamma, seed=seed)


def _tensor_ctx(pb, **opt):
    from paper_2107_00820_gb300 import Context
    return Context(pb.d, pb.n, pb.levels, pb.mu, pb.gamma, mu_eff=pb.meta["mu_eff"], **opt)


def _tensor_oracle(pb, **kw):
    from oracle.mg import Hierarchy
    return Hierarchy(pb.d, pb.n, pb.mu, pb.gamma, kind="tensor", mu_eff=pb.meta["mu_eff"], **kw)


@pytest.mark.parametrize("d,n", [(2, 12), (3, 4)])
def test_tensor_patch_inverses_sampled(d, n):
    pb = _tensor_problem(d, n, 2, 1e2)
    ctx = _tensor_ctx(pb)
    H = _tensor_oracle(pb, smoother="richardson", steps=1)
    m = H.levels[1].mesh
    verts = all_vertices(m)
    NB = 3 ** d
    for vid in list(np.random.default_rng(2).choice(len(verts), size=10, replace=False)) + [0]:
        v = verts[vid]
        cond, idx, Av = _patch_cond(H, 1, v)
        full = ctx.patch_inverse(1, int(vid))
        keep = [a * NB + o for a in range(d) for o in range(NB)
                if np.all((g := 2 * v + (np.array([o % 3, (o // 3) % 3, o // 9][:d]) - 1)) > 0)
                and np.all(g < np.array(m.nn) - 1)]
        got = full[np.ix_(keep, keep)]
        ref = np.linalg.inv(Av)
        assert np.linalg.norm(got - ref) <= max(1e-12, 20 * cond * 2.2e-16) * np.linalg.norm(ref), (vid, cond)


@pytest.mark.parametrize("d,n,levels", [(2, 24, 3), (3, 8, 2)])
def test_tensor_vcycle_fp64(d, n, levels):
    pb = _tensor_problem(d, n, levels, 1e2)
    ctx = _tensor_ctx(pb, sweeps=2)
    H = _tensor_oracle(pb, steps=2)
    b = random_free(H.levels[-1], 3)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    ref = H.vcycle(b)
    cond = _cycle_cond(H, levels - 1, count=20)
    assert rel(host(x), ref) <= max(1e-11, 100 * cond * 2.2e-16), cond


@pytest.mark.parametrize("d,n,levels,gamma", [(2, 24, 3, 1e3), (3, 6, 2, 1e2)])
def test_tensor_solve_fp64_and_mixed(d, n, levels, gamma):
    """Tensor coefficients (C with a contrast of ~1e9).  FP64: the GPU's own patch and
    coarse inverses differ from LAPACK's by cond * eps (cond ~ 1e12 here), which may move
    the step at which rtol is crossed by one; with the oracle's inverses injected into
    the context the iteration count is the oracle's exactly, and the solution matches.
    Mixed: within +2 iterations of FP64 with a true residual that meets rtol, and within
    1e-7 of the converged oracle solution when run on to rtol 1e-11."""
    pb = _tensor_problem(d, n, levels, gamma)
    from oracle.stokes import StokesSolver
    from injection import inject, load_into
    H = _tensor_oracle(pb)
    uo, po, its, _ = StokesSolver(H).solve(pb.f, pb.u_bc, rtol=1e-8)
    ctx = _tensor_ctx(pb, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged and abs(info.iterations - its) <= 1, (info.iterations, its)
    assert rel(u, uo) <= 1e-7 and rel(p, po) <= 1e-5
    load_into(ctx, H, inject(H))
    s = StokesSolver(H)
    uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = ctx.solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its, (info.iterations, its)
    assert _true_residual(s, pb, u, p) <= 1.5e-8
    pb10 = _tensor_problem(d, n, levels, 10.0)
    s10 = StokesSolver(_tensor_oracle(pb10))
    uc, pc, _, _ = s10.solve(pb10.f, pb10.u_bc, rtol=1e-12)
    _, _, i64 = _tensor_ctx(pb10, rtol=1e-8).solve(pb10.f, pb10.u_bc)
    um, pm, im = _tensor_ctx(pb10, rtol=1e-8, mode=A.ALS_MODE_MIXED).solve(pb10.f, pb10.u_bc)
    assert im.converged and im.iterations <= i64.iterations + 2
    assert _true_residual(s10, pb10, um, pm) <= 1.5e-8
    um, pm, im = _tensor_ctx(pb10, rtol=1e-11, mode=A.ALS_MODE_MIXED).solve(pb10.f, pb10.u_bc)
    assert im.converged and rel(um, uc) <= 1e-7 and rel(pm, pc) <= 1e-7, (rel(um, uc), rel(pm, pc))


# --------------------------------------------------------------------------
# P2 (Eq. (P1P2)): W = M_p(1/mu) in the augmentation and S^-1 ~ (1 + gamma) M_p(1/mu)^-1
# --------------------------------------------------------------------------
@pytest.mark.parametrize("d,n", [(2, 8), (3, 4)])
def test_apply_agamma_w_mu_fp64(d, n):
    pb = sinker(d, n, 2, 1e3, dr=1e6, seed=5)
    ctx = context(pb, schur=A.ALS_SCHUR_P2)
    H = oracle(pb, smoother="richardson", steps=1, W="Mp_mu")
    for lvl in range(2):
        lv = H.levels[lvl]
        x = np.random.default_rng(lvl + 7).standard_normal(lv.mesh.nu)
        y = torch.zeros(lv.mesh.nu, dtype=torch.float64, device="cuda")
        ctx.apply_agamma(dev(x), y, lvl)
        assert rel(host(y), lv.A @ x) <= 1e-12


@pytest.mark.parametrize("d,n,levels", [(2, 16, 3), (3, 8, 2)])
def test_solve_p2_fp64_matches_oracle(d, n, levels):
    pb = sinker(d, n, levels, 1e2, dr=1e4, seed=9)
    s = StokesSolver(oracle(pb, W="Mp_mu"), schur="P2")
    uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = context(pb, schur=A.ALS_SCHUR_P2, rtol=1e-8).solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its, (info.iterations, its)
    assert rel(u, uo) <= 1e-8 and rel(p, po) <= 1e-7


def test_mixed_p2_at_extreme_contrast_and_gamma():
    """With W = M_p(1/mu) the AL term scales with mu, so the FP32 V-cycle keeps
    working where the P1 pairing (W = M_p) loses it (gamma / mu_min = 1e7): +2 iterations
    at most, a true residual (oracle) that meets rtol 1e-8, and 1e-7 of the converged oracle
    solution when the mixed solve runs on to rtol 1e-11."""
    pb = sinker(3, 8, 2, 1e3, dr=1e8, seed=11)
    s = StokesSolver(oracle(pb, W="Mp_mu"), schur="P2")
    uc, pc, _, _ = s.solve(pb.f, pb.u_bc, rtol=1e-12)
    _, _, i64 = context(pb, schur=A.ALS_SCHUR_P2, rtol=1e-8).solve(pb.f, pb.u_bc)
    u32, p32, i32 = context(pb, schur=A.ALS_SCHUR_P2, rtol=1e-8, mode=A.ALS_MODE_MIXED).solve(pb.f, pb.u_bc)
    assert i64.converged and i32.converged
    assert i32.iterations <= i64.iterations + 2, (i32.iterations, i64.iterations)
    assert _true_residual(s, pb, u32, p32) <= 1.5e-8
    u11, p11, i11 = context(pb, schur=A.ALS_SCHUR_P2, rtol=1e-11, mode=A.ALS_MODE_MIXED).solve(pb.f, pb.u_bc)
    assert i11.converged and rel(u11, uc) <= 1e-7 and rel(p11, pc) <= 1e-7, (rel(u11, uc), rel(p11, pc))


@pytest.mark.parametrize("d,n,levels,gamma,dr,schur", [(2, 32, 4, 1e2, 1e6, A.ALS_SCHUR_P1),
                                                      (3, 8, 2, 1e3, 1e8, A.ALS_SCHUR_P2)])
def test_mixed_with_fp64_setup(d, n, levels, gamma, dr, schur):
    """options.setup = ALS_SETUP_FP64 keeps the FP32 cycle but computes the patch and
    coarse inverses in FP64: its inverses are the FP64 context's, and it converges with the
    iteration count of the double-float setup (within one), meeting rtol in the oracle's
    true residual, as the double-float setup does."""
    pb = sinker(d, n, levels, gamma, dr, seed=71)
    s = StokesSolver(oracle(pb, W="Mp_mu" if schur == A.ALS_SCHUR_P2 else "Mp"),
                     schur="P2" if schur == A.ALS_SCHUR_P2 else "P1")
    s64 = context(pb, schur=schur, rtol=1e-8)
    df = context(pb, schur=schur, rtol=1e-8, mode=A.ALS_MODE_MIXED)
    f64 = context(pb, schur=schur, rtol=1e-8, mode=A.ALS_MODE_MIXED, setup=A.ALS_SETUP_FP64)
    assert np.array_equal(f64.patch_inverse(levels - 1, 5), s64.patch_inverse(levels - 1, 5))
    _, _, i64 = s64.solve(pb.f, pb.u_bc)
    ud, pd, idf = df.solve(pb.f, pb.u_bc)
    uf, pf, if64 = f64.solve(pb.f, pb.u_bc)
    assert idf.converged and if64.converged and abs(idf.iterations - if64.iterations) <= 1
    assert if64.iterations <= i64.iterations + 2
    for u, p in ((ud, pd), (uf, pf)):
        assert _true_residual(s, pb, u, p) <= 1.5e-8
