"""The order-3 discretisation in three dimensions on the GPU ([Q3]^3 x P2disc, the element of
the 3D sinker runs of Table linear and the k = 3 column of Table k, Sec. 5.2.2) against the
order-k oracle (oracle/qk.py, pinned in 3D on the CPU by tests/test_oracle_qk.py): operator
applies, star inverses (cond-scaled), the smoother, the robust and standard transfers, the
coarse solve and one V-cycle at 1e-12 (FP64) where the arithmetic allows it, FGMRES with the
identical iteration count, the mixed path within +2 iterations and the true residual."""
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
    return P.sinker_problem_k(n, levels, 3, 4, 0.1, 200.0, dr, 10.0, gamma, seed, d=3)


def _ctx(pb, **opt):
    return Context(3, pb.n, pb.levels, pb.mu, pb.gamma, order=3, **opt)


def _oracle(pb, W="Mp", steps=5):
    return HierarchyK(3, pb.n, 3, pb.mu, pb.gamma, steps=steps, W=W)


def _free(lv, seed):
    x = np.random.default_rng(seed).standard_normal(lv.mesh.nu)
    x[lv.bdof] = 0.0
    return x


@pytest.mark.parametrize("schur,W", [(A.ALS_SCHUR_P1, "Mp"), (A.ALS_SCHUR_P2, "Mp_mu")])
def test_q3_3d_apply_fp64(schur, W):
    pb = _problem(4, 2, 1e3, 1e4)
    ctx = _ctx(pb, schur=schur)
    for lvl in range(2):
        lv = LevelK(3, pb.level_n[lvl], 3, pb.mu[lvl], pb.gamma, W)
        x = np.random.default_rng(lvl).standard_normal(lv.mesh.nu)   # boundary entries too
        y = torch.zeros(lv.mesh.nu, dtype=torch.float64, device="cuda")
        ctx.apply_agamma(dev(x), y, lvl)
        assert rel(host(y), lv.A @ x) <= 1e-12


def test_q3_3d_apply_fp32_and_stokes_operator():
    pb = _problem((4, 6, 4), 2, 1e2, 1e3)   # unequal cell counts: the axis orders must agree
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


def test_q3_3d_star_inverses_sampled():
    pb = _problem(4, 2, 1e2, 1e4)
    ctx = _ctx(pb)
    lv = LevelK(3, pb.n, 3, pb.mu[1], pb.gamma)
    m = lv.mesh
    verts = all_vertices_k(m)
    offs = np.array([[o % 5, (o // 5) % 5, o // 25] for o in range(125)]) - 2
    centre = int(np.flatnonzero(np.all(verts == 2, axis=1))[0])   # interior: all 375 dofs free
    picks = list(np.random.default_rng(6).choice(len(verts), 6, replace=False)) + [0, len(verts) - 1, centre]
    for vid in picks:
        v = verts[vid]
        idx = star_dofs_k(m, v)
        Av = lv.A[idx][:, idx].toarray()
        g = 3 * v + offs
        free = np.all(g > 0, axis=1) & np.all(g < np.array(m.nn) - 1, axis=1)
        keep = [a * 125 + o for a in range(3) for o in range(125) if free[o]]
        assert len(keep) == len(idx)
        full = ctx.patch_inverse(1, int(vid))
        ref = np.linalg.inv(Av)
        cond = np.linalg.cond(Av)
        assert np.linalg.norm(full[np.ix_(keep, keep)] - ref) <= max(1e-12, 20 * cond * 2.2e-16) * np.linalg.norm(ref)
        other = np.setdiff1d(np.arange(375), keep)
        assert np.allclose(full[np.ix_(other, other)], np.eye(len(other)))


def test_q3_3d_star_inverses_double_float():
    """Mixed mode eliminates the 3D stars in double-float (unit roundoff 2^-48): the inverses
    stay within the a-priori bound of elimination, n cond u (n = 375 pivots, u = 2^-48),
    of the oracle's; ALS_SETUP_FP64 meets the FP64 form of the same bound, and the
    double-float error is the larger one (it is the arithmetic, not the assembly)."""
    pb = _problem(4, 2, 1e3, 1e6)
    lv = LevelK(3, pb.n, 3, pb.mu[1], pb.gamma)
    verts = all_vertices_k(lv.mesh)
    vid = int(np.flatnonzero(np.all(verts == 2, axis=1))[0])
    idx = star_dofs_k(lv.mesh, verts[vid])
    Av = lv.A[idx][:, idx].toarray()
    ref = np.linalg.inv(Av)
    cond = np.linalg.cond(Av)
    errs = {}
    for setup, eps in ((A.ALS_SETUP_AUTO, 2.0 ** -48), (A.ALS_SETUP_FP64, 2.0 ** -53)):
        full = _ctx(pb, mode=A.ALS_MODE_MIXED, setup=setup).patch_inverse(1, vid)
        errs[setup] = np.linalg.norm(full - ref) / np.linalg.norm(ref)
        assert errs[setup] <= 375 * cond * eps, (setup, errs[setup], cond)
    assert errs[A.ALS_SETUP_FP64] < errs[A.ALS_SETUP_AUTO], errs


@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_q3_3d_star_smoother(prec):
    pb = _problem(4, 2, 1e2, 1e3)
    ctx = _ctx(pb)
    lv = LevelK(3, pb.n, 3, pb.mu[1], pb.gamma)
    r = _free(lv, 7)
    dt = torch.float64 if prec == A.ALS_PREC_FP64 else torch.float32
    z = torch.zeros(lv.mesh.nu, dtype=dt, device="cuda")
    ctx.star_smooth(1, dev(r, dt), z, prec)
    assert rel(host(z), star_patches_k(lv).apply(r)) <= (1e-11 if prec == A.ALS_PREC_FP64 else 1e-4)


@pytest.mark.parametrize("transfer", [A.ALS_TRANSFER_ROBUST, A.ALS_TRANSFER_STANDARD])
def test_q3_3d_transfers(transfer):
    pb = _problem(4, 2, 1e2, 1e3)
    ctx = _ctx(pb, transfer=transfer)
    c = LevelK(3, pb.level_n[0], 3, pb.mu[0], pb.gamma)
    f = LevelK(3, pb.n, 3, pb.mu[1], pb.gamma)
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


def test_q3_3d_coarse_solve():
    pb = _problem(4, 2, 1e2, 1e4)
    ctx = _ctx(pb)
    H = _oracle(pb)
    b = _free(H.levels[0], 10)
    x = torch.zeros_like(dev(b))
    ctx.coarse_solve(dev(b), x)
    f = H.coarse_free
    cond = np.linalg.cond(H.levels[0].A.toarray()[np.ix_(f, f)])
    assert rel(host(x), H.coarse_solve(b)) <= max(1e-12, 10 * cond * 2.2e-16)


@pytest.mark.parametrize("n,levels", [(4, 2), (8, 3)])
def test_q3_3d_vcycle_fp64(n, levels):
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
def test_q3_3d_cycle_variants_fp64(smoother, cycle):
    """The F-cycle (the paper's cycle for Table linear) and Richardson smoothing (damping
    2^-d) at order 3, against the order-k oracle's cycles."""
    pb = _problem(8, 3, 1.0, 1e2)
    ctx = _ctx(pb, sweeps=2, smoother=smoother, cycle=cycle)
    H = HierarchyK(3, pb.n, 3, pb.mu, pb.gamma, steps=2,
                   smoother="gmres" if smoother == A.ALS_SMOOTH_GMRES else "richardson",
                   cycle="F" if cycle == A.ALS_CYCLE_F else "V")
    b = _free(H.levels[-1], 12)
    x = torch.zeros_like(dev(b))
    ctx.vcycle(dev(b), x)
    assert rel(host(x), H.cycle(b)) <= 1e-12


@pytest.mark.parametrize("schur,W,gamma,dr", [(A.ALS_SCHUR_P1, "Mp", 1e2, 1e4), (A.ALS_SCHUR_P2, "Mp_mu", 1e3, 1e6)])
def test_q3_3d_fgmres_counts_equal_the_oracle(schur, W, gamma, dr):
    pb = _problem(8, 3, gamma, dr)
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


def test_q3_3d_loaded_inverses_give_the_same_fp32_smoother():
    """Caller-supplied FP64 inverses (packed by diagonals) are rounded into the FP32 wrapped
    rows by the same rule as the setup's: reloading the context's own inverses leaves the
    FP32 smoother's output bit for bit unchanged, and loading the oracle's inverses gives the
    oracle's smoother within FP32 rounding."""
    pb = _problem(4, 2, 1e2, 1e3)
    ctx = _ctx(pb)
    lv = LevelK(3, pb.n, 3, pb.mu[1], pb.gamma)
    nverts = 5 ** 3
    np_ = 375
    stride = (np_ * (np_ + 1) // 2 + 3) // 4 * 4
    starts = [t * np_ - t * (t - 1) // 2 for t in range(np_)]

    def pack(full):
        return np.concatenate([np.diag(full, t) for t in range(np_)] + [np.zeros(stride - starts[-1] - 1)])

    r = dev(_free(lv, 13), torch.float32)
    z0 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z0, A.ALS_PREC_FP32)
    own = np.concatenate([pack(ctx.patch_inverse(1, v)) for v in range(nverts)])
    ctx.load_patch_inverses(1, own)
    z1 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z1, A.ALS_PREC_FP32)
    assert torch.equal(z0, z1)
    m = lv.mesh
    verts = all_vertices_k(m)
    offs = np.array([[o % 5, (o // 5) % 5, o // 25] for o in range(125)]) - 2
    packs = []
    for v in verts:
        idx = star_dofs_k(m, v)
        g = 3 * v + offs
        free = np.all(g > 0, axis=1) & np.all(g < np.array(m.nn) - 1, axis=1)
        keep = [a * 125 + o for a in range(3) for o in range(125) if free[o]]
        full = np.eye(np_)
        full[np.ix_(keep, keep)] = np.linalg.inv(lv.A[idx][:, idx].toarray())
        packs.append(pack(0.5 * (full + full.T)))
    ctx.load_patch_inverses(1, np.concatenate(packs))
    z2 = torch.zeros_like(r)
    ctx.star_smooth(1, r, z2, A.ALS_PREC_FP32)
    assert rel(host(z2), star_patches_k(lv).apply(host(r).astype(np.float64))) <= 1e-5


@pytest.mark.parametrize("mode", [A.ALS_MODE_FP64, A.ALS_MODE_MIXED])
def test_q3_batch_of_orders_and_dimensions(mode):
    """A batch mixing order-3 instances in 2D and 3D with an order-2 one: the merged form
    refuses order 3 (its kernels are order 2), the batch runs the instances' own cycle
    graphs side by side, and every instance is bitwise its single-instance solve."""
    from paper_2107_00820_gb300 import Batch
    opts = {"mode": mode, "schur": A.ALS_SCHUR_P2, "rtol": 1e-8, "order": 3}
    pbs = [_problem(4, 2, 1e2, 1e4, seed=41), _problem(8, 3, 1e3, 1e4, seed=42),
           P.sinker_problem_k(16, 3, 3, 4, 0.1, 200.0, 1e4, 10.0, 1e2, 43, d=2)]
    ins = [{"dim": pb.d, "n": pb.n, "levels": pb.levels, "coeffs": pb.mu, "gamma": pb.gamma, "options": opts}
           for pb in pbs]
    pb2 = P.sinker_problem(2, 16, 3, 4, 0.1, 200.0, 1e4, 10.0, 1e2, 44)
    opts2 = dict(opts, order=2)
    ins.append({"dim": 2, "n": pb2.n, "levels": pb2.levels, "coeffs": pb2.mu, "gamma": pb2.gamma, "options": opts2})
    batch = Batch(ins)
    assert batch.mode == A.ALS_BATCH_BRANCHES
    ub, pb_, infos = batch.solve([pb.f for pb in pbs] + [pb2.f], [pb.u_bc for pb in pbs] + [pb2.u_bc])
    for i, (pb, o) in enumerate(zip(pbs + [pb2], [opts] * 3 + [opts2])):
        ctx = Context(pb.d, pb.n, pb.levels, pb.mu, pb.gamma, **o)
        u, p, info = ctx.solve(pb.f, pb.u_bc)
        assert infos[i].converged == 1 and infos[i].iterations == info.iterations
        assert np.array_equal(ub[i], u) and np.array_equal(pb_[i], p)
        ctx.close()
    batch.close()


def _to_bfloat16(x):
    """Round to the nearest bfloat16 (8 significant bits), ties to even, from float64."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def test_q3_3d_smoother_with_bfloat16_rows():
    """ALS_STORE_BF16 at order 3 in 3D: the FP32 smoother streams the wrapped rows rounded
    to bfloat16 from the FP64 inverses; against the star products of the context's own FP64
    inverses rounded the same way (host, FP64 sums), entry by entry within FP32 rounding of
    the sums, and visibly different from the FP32-stored smoother (the rounding is real)."""
    pb = _problem(4, 2, 1e2, 1e3)
    ctx = _ctx(pb, store=A.ALS_STORE_BF16)
    ref32 = _ctx(pb)
    lv = LevelK(3, pb.n, 3, pb.mu[1], pb.gamma)
    m = lv.mesh
    r = _free(lv, 14).astype(np.float32).astype(np.float64)
    z = torch.zeros(m.nu, dtype=torch.float32, device="cuda")
    ctx.star_smooth(1, dev(r, torch.float32), z, A.ALS_PREC_FP32)
    z32 = torch.zeros_like(z)
    ref32.star_smooth(1, dev(r, torch.float32), z32, A.ALS_PREC_FP32)
    verts = all_vertices_k(m)
    offs = np.array([[o % 5, (o // 5) % 5, o // 25] for o in range(125)]) - 2
    ref, scale = np.zeros(m.nu), np.zeros(m.nu)
    for vid, v in enumerate(verts):
        g = 3 * v + offs
        free = np.all(g > 0, axis=1) & np.all(g < np.array(m.nn) - 1, axis=1)
        nodes = (g[:, 0] + m.nn[0] * (g[:, 1] + m.nn[1] * g[:, 2]))
        dofs = np.concatenate([a * m.N + nodes for a in range(3)])
        keep = np.flatnonzero(np.tile(free, 3))
        F = _to_bfloat16(ctx.patch_inverse(1, vid))[np.ix_(keep, keep)]
        rv = r[dofs[keep]]
        np.add.at(ref, dofs[keep], F @ rv)
        np.add.at(scale, dofs[keep], np.abs(F) @ np.abs(rv))
    got = host(z)
    assert np.all(np.abs(got - ref) <= 400 * 2.0 ** -24 * scale + 1e-30)
    assert rel(host(z32), ref) > 1e-4          # the FP32-stored smoother differs by the rounding


def test_q3_3d_mixed_solve_with_bfloat16_rows():
    """The mixed solve on bfloat16 rows at mild contrast: converges (P2 pairing), a few
    iterations more than on FP32 rows at most."""
    pb = _problem(8, 3, 1e2, 1e4)
    kw = dict(schur=A.ALS_SCHUR_P2, rtol=1e-8, mode=A.ALS_MODE_MIXED)
    _, _, i32 = _ctx(pb, **kw).solve(pb.f, pb.u_bc)
    _, _, i16 = _ctx(pb, store=A.ALS_STORE_BF16, **kw).solve(pb.f, pb.u_bc)
    assert i32.converged and i16.converged
    assert i16.iterations <= i32.iterations + 4, (i16.iterations, i32.iterations)
