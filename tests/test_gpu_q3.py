"""The order-3 discretisation on the GPU ([Q3]^2 x P2disc, the higher-order study of
Sec. 5.2.2, Table k) against the order-k oracle (oracle/qk.py, pinned on the CPU by
tests/test_oracle_qk.py): every stage of the path at 1e-12 (FP64) where the arithmetic
allows it -- operator applies, star inverses (cond-scaled), the smoother, the robust and
standard transfers, the coarse solve, one V-cycle -- and FGMRES with the identical
iteration count; the mixed path within its FP32 rounding and +2 iterations."""
import numpy as np
import pytest

from gpu_helpers import dev, host, rel, torch  # noqa: F401
from oracle.qk import (HierarchyK, LevelK, all_vertices_k, robust_prolongation_k, standard_prolongation_k,
                       star_dofs_k, star_patches_k)
from oracle.stokes import StokesSolver
from synthetic import problems as P

from paper_2107_00820_gb300 import Context, alstokes as A  # noqa: E402

pytestmark = pytest.mark.gpu


def _problem(n, levels, gamma, dr, seed=3):
    return P.sinker_problem_k(n, levels, 3, 4, 0.1, 200.0, dr, 10.0, gamma, seed)


def _ctx(pb, **opt):
    return Context(2, pb.n, pb.levels, pb.mu, pb.gamma, order=3, **opt)


def _oracle(pb, W="Mp", steps=5):
    return HierarchyK(2, pb.n, 3, pb.mu, pb.gamma, steps=steps, W=W)


def _free(lv, seed):
    x = np.random.default_rng(seed).standard_normal(lv.mesh.nu)
    x[lv.bdof] = 0.0
    return x


@pytest.mark.parametrize("schur,W", [(A.ALS_SCHUR_P1, "Mp"), (A.ALS_SCHUR_P2, "Mp_mu")])
def test_q3_apply_fp64(schur, W):
    pb = _problem(8, 2, 1e3, 1e4)
    ctx = _ctx(pb, schur=schur)
    for lvl in range(2):
        lv = LevelK(2, pb.level_n[lvl], 3, pb.mu[lvl], pb.gamma, W)
        x = np.random.default_rng(lvl).standard_normal(lv.mesh.nu)   # boundary entries too
        y = torch.zeros(lv.mesh.nu, dtype=torch.float64, device="cuda")
        ctx.apply_agamma(dev(x), y, lvl)
        assert rel(host(y), lv.A @ x) <= 1e-12


def test_q3_apply_fp32_and_stokes_operator():
    pb = _problem(8, 2, 1e2, 1e3)
    ctx = _ctx(pb)
    H = _oracle(pb)
    lv = H.levels[-1]
    x = np.random.default_rng(4).standard_normal(lv.mesh.nu)
    y = torch.zeros(lv.mesh.nu, dtype=torch.float32, device="cuda")
    ctx.apply_agamma(dev(x, torch.float32), y, 1, A.ALS_PREC_FP32)
    assert rel(host(y), lv.A @ x.astype(np.float32).astype(np.float64)) <= 2e-5
    s = StokesSolver(H)
    rng = np.random.default_rng(5)
    u, p = rng.standard_normal(s.nu), rng.standard_normal(s.np_)
    yu = torch.zeros(s.nu, dtype=torch.float64, device="cuda")
    yp = torch.zeros(s.np_, dtype=torch.float64, device="cuda")
    ctx.apply_stokes(dev(u), dev(p), yu, yp)
    ref = s.matvec(np.concatenate([u, p]))
    assert rel(host(yu), ref[: s.nu]) <= 1e-12 and rel(host(yp), ref[s.nu:]) <= 1e-12


def test_q3_star_inverses_sampled():
    pb = _problem(8, 2, 1e2, 1e4)
    ctx = _ctx(pb)
    lv = LevelK(2, pb.n, 3, pb.mu[1], pb.gamma)
    m = lv.mesh
    verts = all_vertices_k(m)
    offs = np.array([[o % 5, o // 5] for o in range(25)]) - 2
    for vid in list(np.random.default_rng(6).choice(len(verts), 10, replace=False)) + [0, len(verts) - 1]:
        v = verts[vid]
        idx = star_dofs_k(m, v)
        Av = lv.A[idx][:, idx].toarray()
        g = 3 * v + offs
        free = np.all(g > 0, axis=1) & np.all(g < np.array(m.nn) - 1, axis=1)
        keep = [a * 25 + o for a in range(2) for o in range(25) if free[o]]
        assert len(keep) == len(idx)
        full = ctx.patch_inverse(1, int(vid))
        ref = np.linalg.inv(Av)
        cond = np.linalg.cond(Av)
        assert np.linalg.norm(full[np.ix_(keep, keep)] - ref) <= max(1e-12, 20 * cond * 2.2e-16) * np.linalg.norm(ref)
        other = np.setdiff1d(np.arange(50), keep)
        assert np.allclose(full[np.ix_(other, other)], np.eye(len(other)))


@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_q3_star_smoother(prec):
    pb = _problem(8, 2, 1e2, 1e3)
    ctx = _ctx(pb)
    lv = LevelK(2, pb.n, 3, pb.mu[1], pb.gamma)
    r = _free(lv, 7)
    dt = torch.float64 if prec == A.ALS_PREC_FP64 else torch.float32
    z = torch.zeros(lv.mesh.nu, dtype=dt, device="cuda")
    ctx.star_smooth(1, dev(r, dt), z, prec)
    assert rel(host(z), star_patches_k(lv).apply(r)) <= (1e-11 if prec == A.ALS_PREC_FP64 else 1e-4)


@pytest.mark.parametrize("transfer", [A.ALS_TRANSFER_ROBUST, A.ALS_TRANSFER_STANDARD])
def test_q3_transfers(transfer):
    pb = _problem(8, 2, 1e2, 1e3)
    ctx = _ctx(pb, transfer=transfer)
    c = LevelK(2, pb.level_n[0], 3, pb.mu[0], pb.gamma)
    f = LevelK(2, pb.n, 3, pb.mu[1], pb.gamma)
    P_ = robust_prolongation_k(c.mesh, f)[0] if transfer == A.ALS_TRANSFER_ROBUST else \
        standard_prolongation_k(c.mesh, f.mesh)
    xc = _free(c, 8)
    xf = torch.zeros(f.mesh.nu, dtype=torch.float64, device="cuda")
    ctx.prolong(1, dev(xc), xf)
    assert rel(host(xf), P_ @ xc) <= 1e-11
    rf = _free(f, 9)
    rc = torch.zeros(c.mesh.nu, dtype=torch.float64, device="cuda")
    ctx.restrict(1, dev(rf), rc)
    assert rel(host(rc), P_.T @ rf) <= 1e-11


def test_q3_coarse_solve():
    pb = _problem(8, 2, 1e2, 1e4)
    ctx = _ctx(pb)
    H = _oracle(pb)
    b = _free(H.levels[0], 10)
    x = torch.zeros_like(dev(b))
    ctx.coarse_solve(dev(b), x)
    f = H.coarse_free
    cond = np.linalg.cond(H.levels[0].A.toarray()[np.ix_(f, f)])
    assert rel(host(x), H.coarse_solve(b)) <= max(1e-12, 10 * cond * 2.2e-16)


@pytest.mark.parametrize("n,levels", [(8, 2), (16, 3)])
def test_q3_vcycle_fp64(n, levels):
    pb = _problem(n, levels, 1.0, 1e2)
    ctx = _ctx(pb, sweeps=2)
    H = _oracle(pb, steps=2)
    b = _free(H.levels[-1], 11)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.vcycle(b)) <= 1e-12


@pytest.mark.parametrize("smoother,cycle", [(A.ALS_SMOOTH_GMRES, A.ALS_CYCLE_F),
                                           (A.ALS_SMOOTH_RICHARDSON, A.ALS_CYCLE_V),
                                           (A.ALS_SMOOTH_RICHARDSON, A.ALS_CYCLE_F)])
def test_q3_cycle_variants_fp64(smoother, cycle):
    """The F-cycle (the paper's cycle for Table linear) and Richardson smoothing (damping
    2^-d) at order 3, against the order-k oracle's cycles."""
    pb = _problem(16, 3, 1.0, 1e2)
    ctx = _ctx(pb, sweeps=2, smoother=smoother, cycle=cycle)
    H = HierarchyK(2, pb.n, 3, pb.mu, pb.gamma, steps=2,
                   smoother="gmres" if smoother == A.ALS_SMOOTH_GMRES else "richardson",
                   cycle="F" if cycle == A.ALS_CYCLE_F else "V")
    b = _free(H.levels[-1], 12)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.cycle(b)) <= 1e-12


@pytest.mark.parametrize("schur,W,gamma,dr", [(A.ALS_SCHUR_P1, "Mp", 1e2, 1e4), (A.ALS_SCHUR_P2, "Mp_mu", 1e3, 1e6)])
def test_q3_fgmres_counts_equal_the_oracle(schur, W, gamma, dr):
    pb = _problem(16, 3, gamma, dr)
    s = StokesSolver(_oracle(pb, W=W), schur="P2" if W == "Mp_mu" else "P1")
    uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-8)
    u, p, info = _ctx(pb, schur=schur, rtol=1e-8).solve(pb.f, pb.u_bc)
    assert info.converged and info.iterations == its, (info.iterations, its)
    assert rel(u, uo) <= 1e-9 and rel(p, po) <= 1e-8, (rel(u, uo), rel(p, po))
    # mixed precision: +2 iterations at most, the true residual meets rtol
    from test_gpu_parity import _true_residual
    um, pm, im = _ctx(pb, schur=schur, rtol=1e-8, mode=A.ALS_MODE_MIXED).solve(pb.f, pb.u_bc)
    assert im.converged and im.iterations <= its + 2, (im.iterations, its)
    assert _true_residual(s, pb, um, pm) <= 1.5e-8


def test_q3_loaded_inverses_give_the_same_fp32_smoother():
    """Caller-supplied FP64 inverses (packed by diagonals) are rounded into the FP32 wrapped
    rows by the setup's own rule: reloading the context's inverses leaves the FP32
    smoother's output bit for bit unchanged."""
    pb = _problem(8, 2, 1e2, 1e3)
    ctx = _ctx(pb)
    lv = LevelK(2, pb.n, 3, pb.mu[1], pb.gamma)
    np_ = 50
    stride = (np_ * (np_ + 1) // 2 + 3) // 4 * 4
    starts = [t * np_ - t * (t - 1) // 2 for t in range(np_)]

    def pack(full):
        return np.concatenate([np.diag(full, t) for t in range(np_)] + [np.zeros(stride - starts[-1] - 1)])

    r = dev(_free(lv, 13), torch.float32)
    z0 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z0, A.ALS_PREC_FP32)
    ctx.load_patch_inverses(1, np.concatenate([pack(ctx.patch_inverse(1, v)) for v in range(9 ** 2)]))
    z1 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z1, A.ALS_PREC_FP32)
    assert torch.equal(z0, z1)


def test_q3_fp32_star_kernel_with_warps_walking_several_stars():
    """The FP32 star kernel is persistent (three blocks an SM; each warp walks several stars,
    the next star's rows prefetched while it multiplies the current one).  On 2D 96^2
    (9,409 stars, more than the 3,648 warps of a 152-SM grid; 2,304 interior stars for the
    transfers) the FP32 smoother and the FP32 robust transfers, whose local solves write and
    subtract through the same kernel, match the FP64 path (its own star kernel) within the
    FP32 smoother bar: a star skipped, repeated or read from another warp's rows fails it."""
    pb = _problem(96, 5, 1.0, 1e2)
    ctx = _ctx(pb)
    L = pb.levels - 1
    rng = np.random.default_rng(23)
    out = {}
    r = rng.standard_normal(ctx.nu(L))
    xc = rng.standard_normal(ctx.nu(L - 1))
    for prec, dt in ((A.ALS_PREC_FP64, torch.float64), (A.ALS_PREC_FP32, torch.float32)):
        z = torch.zeros(ctx.nu(L), dtype=dt, device="cuda")
        ctx.star_smooth(L, dev(r, dt), z, prec)
        xf = torch.zeros(ctx.nu(L), dtype=dt, device="cuda")
        ctx.prolong(L, dev(xc, dt), xf, prec)
        rc = torch.zeros(ctx.nu(L - 1), dtype=dt, device="cuda")
        ctx.restrict(L, dev(r, dt), rc, prec)
        out[prec] = [host(z), host(xf), host(rc)]
    for a, b in zip(out[A.ALS_PREC_FP32], out[A.ALS_PREC_FP64]):
        assert rel(a, b) <= 1e-4
