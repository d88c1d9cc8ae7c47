"""Parity at the benchmark's full sizes, in the configuration bench.py times.

Every workload of bench.py (3D sinker 32^3 hexes with 4 levels, DR 1e8, gamma 10, and the
same at gamma 1e4 with the P2 pairing; 2D sinker 128^2 quads with 5 levels, DR 1e6, gamma
1e2; 3D viscoplastic 48^3 hexes with the 21-entry tensor, gamma 1e3, P2 pairing) is built at full size into a mixed-mode context
with the benchmark's options (5 smoothing steps, FGMRES to 1e-8, at most 200 iterations).
The oracle cannot assemble these meshes in test time, so each stage's output is sampled
and every sampled entry is recomputed from the cells it depends on
(tests/local_oracle.py, itself checked entry for entry against the assembled oracle on
small meshes), with elementwise bounds scaled by the sum of the absolute values of the
terms (rounding of any summation order) and, where a patch inverse enters, by
cond(A_v) 2^-48 (the double-float inversion).  The solves are checked by properties that
hold at any size: the true residual of the mixed solution, evaluated cell by cell by the
oracle, and the mixed solve against the all-FP64 GPU solve.

Bounds: FP64 stages 1e-12 of the sum of |terms|; FP32 stages 400 (smoother: one
81-term product per star and a gather of at most 8) or 1000 (operator apply and
transfers: products of sum-factorised quadrature sums) FP32 unit roundoffs of it; plus
100 cond(A_v) 2^-48 ||A_v^-1|| ||r_v|| wherever a patch inverse enters.  A wrong index,
sign, layout or dropped term gives an error of order the sum itself.

The file name sorts last so that the other GPU tests run first."""
import numpy as np
import pytest

import bench
from gpu_helpers import dev, host, torch  # noqa: F401
from local_oracle import LocalLevel, LocalTransfer, stokes_residual
from oracle.fem import Level

from paper_2107_00820_gb300 import Context, alstokes as A  # noqa: E402

pytestmark = pytest.mark.gpu

U_DF = 2.0 ** -48          # unit roundoff of the double-float patch and coarse inversions
EPS32 = 2.0 ** -24


class Full:
    """A workload at full size: problem, mixed context, cell-local oracle levels."""

    def __init__(self, name):
        spec = bench.WORKLOADS[name]
        self.name, self.spec = name, spec
        self.pb = pb = bench.make_problem(spec)
        self.d, self.L = pb.d, pb.levels
        self.tensor = spec.get("kind") == "tensor"
        self.kind = "tensor" if self.tensor else "scalar"
        self.W = "Mp_mu" if spec.get("schur") == "P2" else "Mp"
        self.schur = A.ALS_SCHUR_P2 if spec.get("schur") == "P2" else A.ALS_SCHUR_P1
        self.mu_eff = pb.meta["mu_eff"] if self.tensor else None
        self.opts = dict(rtol=bench.RTOL, maxit=200, sweeps=spec["sweeps"], schur=self.schur)
        self.ctx = Context(pb.d, pb.n, pb.levels, pb.mu, pb.gamma, mu_eff=self.mu_eff,
                           mode=A.ALS_MODE_MIXED, **self.opts)
        self.sizes = pb.level_n
        self._local = {}

    def local(self, lvl):
        if lvl not in self._local:
            self._local[lvl] = LocalLevel(self.d, self.sizes[lvl], self.pb.mu[lvl], self.pb.gamma,
                                          kind=self.kind,
                                          mu_eff=None if self.mu_eff is None else self.mu_eff[lvl],
                                          W=self.W)
        return self._local[lvl]

    def nu(self, lvl):
        return self.d * int(np.prod([2 * v + 1 for v in self.sizes[lvl]]))

    def random_free(self, lvl, seed):
        lv = self.local(lvl)
        x = np.random.default_rng(seed).standard_normal(lv.m.nu)
        x[~lv.free_dof] = 0.0
        return x

    def sample_dofs(self, lvl, seed, count):
        """Half uniform over the level's dofs, half at nodes within two node
        spacings of the boundary (boundary rows, truncated stars, corner cells)."""
        lv = self.local(lvl)
        rng = np.random.default_rng(seed)
        nodes = lv.m.nodes
        near = np.flatnonzero(np.any((nodes <= 2) | (nodes >= lv.nn - 3), axis=1))
        a = rng.integers(0, self.d, count)
        pick = np.concatenate([rng.integers(0, lv.m.N, count // 2), rng.choice(near, count - count // 2)])
        return np.unique(a * lv.m.N + pick)

    def sample_vertices(self, lvl, seed, count):
        """Every corner, vertices on faces and edges, and uniform interior ones."""
        n = np.array(self.sizes[lvl])
        rng = np.random.default_rng(seed)
        out = [np.array(c) * n for c in np.ndindex(*(2,) * self.d)]
        for _ in range(count):
            v = rng.integers(0, n + 1)
            k = rng.integers(0, self.d)
            if rng.random() < 0.5:
                v[k] = rng.choice([0, n[k]])
            out.append(v)
        return out

    def close(self):
        self.ctx.close()


# the workloads the benchmark has timed on a GPU first, then the 2D one
@pytest.fixture(scope="module", params=["sinker3d_32", "viscoplastic3d_48", "sinker2d_128", "sinker3d_32_g1e4"])
def full(request):
    f = Full(request.param)
    yield f
    f.close()
    torch.cuda.empty_cache()


def _finest(full):
    return full.L - 1


def test_apply_agamma_sampled(full):
    """a1/a2 at full size: FP64 apply within 1e-12 of the oracle rows, FP32 within its
    rounding, both elementwise against the sum of |terms|."""
    lvl = _finest(full)
    lv = full.local(lvl)
    x = full.random_free(lvl, 1)
    dofs = full.sample_dofs(lvl, 2, 160)
    y = torch.zeros(lv.m.nu, dtype=torch.float64, device="cuda")
    full.ctx.apply_agamma(dev(x), y, lvl, A.ALS_PREC_FP64)
    ref, scale = lv.apply_rows(x, dofs)
    got = host(y)[dofs]
    err = np.abs(got - ref)
    assert np.all(err <= 1e-12 * scale + 1e-300), np.max(err / np.maximum(scale, 1e-300))
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = torch.zeros(lv.m.nu, dtype=torch.float32, device="cuda")
    full.ctx.apply_agamma(dev(x32, torch.float32), y32, lvl, A.ALS_PREC_FP32)
    ref32, scale32 = lv.apply_rows(x32, dofs)
    got32 = host(y32)[dofs]
    err32 = np.abs(got32 - ref32)
    assert np.all(err32 <= 1000 * EPS32 * scale32 + 1e-300), np.max(err32 / np.maximum(scale32, 1e-300))


@pytest.mark.parametrize("below", [0, 1])
def test_patch_inverses_sampled(full, below):
    """a3 at full size: the double-float inverses of sampled vertex stars (corners,
    faces, edges, interior) of the two finest levels against LAPACK on the locally
    assembled star matrix; identity rows at absent and boundary nodes."""
    lvl = _finest(full) - below
    lv = full.local(lvl)
    n = np.array(full.sizes[lvl])
    strides = np.cumprod(np.concatenate([[1], n[:-1] + 1]))
    for v in full.sample_vertices(lvl, 10 + below, 10):
        vid = int((v * strides).sum())
        got = full.ctx.patch_inverse(lvl, vid)
        inv, keep, _, cond = lv.patch_inverse(v)
        err = np.linalg.norm(got[np.ix_(keep, keep)] - inv) / np.linalg.norm(inv)
        assert err <= max(1e-13, 100 * cond * U_DF), (tuple(v), cond, err)
        other = np.setdiff1d(np.arange(got.shape[0]), keep)
        if len(other):
            assert np.allclose(got[np.ix_(other, other)], np.eye(len(other)))
            assert np.abs(got[np.ix_(keep, other)]).max() <= 1e-12 * np.abs(inv).max()


def test_star_smoother_sampled(full):
    """a4 at full size: z = sum_v I_v A_v^-1 I_v^T r on the finest level, FP64 and FP32
    (the benchmark's cycle precision), at sampled dofs."""
    lvl = _finest(full)
    lv = full.local(lvl)
    r = full.random_free(lvl, 3)
    dofs = full.sample_dofs(lvl, 4, 60)
    z = torch.zeros(lv.m.nu, dtype=torch.float64, device="cuda")
    full.ctx.star_smooth(lvl, dev(r), z, A.ALS_PREC_FP64)
    ref, absum, cscale = lv.smooth_rows(r, dofs)
    err = np.abs(host(z)[dofs] - ref)
    assert np.all(err <= 1e-12 * absum + 100 * U_DF * cscale + 1e-300), np.max(err / np.maximum(absum, 1e-300))
    r32 = r.astype(np.float32).astype(np.float64)
    z32 = torch.zeros(lv.m.nu, dtype=torch.float32, device="cuda")
    full.ctx.star_smooth(lvl, dev(r32, torch.float32), z32, A.ALS_PREC_FP32)
    ref32, absum32, cscale32 = lv.smooth_rows(r32, dofs)
    err32 = np.abs(host(z32)[dofs] - ref32)
    bound32 = 400 * EPS32 * absum32 + 100 * U_DF * cscale32
    assert np.all(err32 <= bound32 + 1e-300), np.max(err32 / np.maximum(absum32, 1e-300))


@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_transfers_sampled(full, prec):
    """a5/a6 at full size: P~ into the finest level and P~^T out of it, at sampled
    fine and coarse dofs (nodes inside and on the boundaries of coarse cells)."""
    lvl = _finest(full)
    T = LocalTransfer(full.local(lvl - 1), full.local(lvl))
    fp64 = prec == A.ALS_PREC_FP64
    dt = torch.float64 if fp64 else torch.float32
    rnd = (lambda a: a) if fp64 else (lambda a: a.astype(np.float32).astype(np.float64))
    tol = 1e-12 if fp64 else 1000 * EPS32
    ec = rnd(full.random_free(lvl - 1, 5))
    xf = torch.zeros(full.nu(lvl), dtype=dt, device="cuda")
    full.ctx.prolong(lvl, dev(ec, dt), xf, prec)
    dofs = full.sample_dofs(lvl, 6, 40)
    ref, absum, cscale = T.prolong_rows(ec, dofs)
    err = np.abs(host(xf)[dofs] - ref)
    assert np.all(err <= tol * absum + 100 * U_DF * cscale + 1e-300), np.max(err / np.maximum(absum, 1e-300))
    rf = rnd(full.random_free(lvl, 7))
    rc = torch.zeros(full.nu(lvl - 1), dtype=dt, device="cuda")
    full.ctx.restrict(lvl, dev(rf, dt), rc, prec)
    cdofs = full.sample_dofs(lvl - 1, 8, 24)
    ref, absum, cscale = T.restrict_rows(rf, cdofs)
    err = np.abs(host(rc)[cdofs] - ref)
    assert np.all(err <= tol * absum + 100 * U_DF * cscale + 1e-300), np.max(err / np.maximum(absum, 1e-300))


def test_coarse_solve(full):
    """a7 at full size: the coarsest level is small enough for the assembled oracle;
    the double-float inverse applied in FP64 meets the dense solve within a small
    multiple of cond 2^-48."""
    pb = full.pb
    lv0 = Level(full.d, full.sizes[0], pb.mu[0], pb.gamma, full.kind,
                None if full.mu_eff is None else full.mu_eff[0], full.W)
    b = np.random.default_rng(9).standard_normal(lv0.mesh.nu)
    b[lv0.bdof] = 0.0
    x = torch.zeros(lv0.mesh.nu, dtype=torch.float64, device="cuda")
    full.ctx.coarse_solve(dev(b), x, A.ALS_PREC_FP64)
    fr = np.flatnonzero(lv0.free)
    A0 = lv0.A.toarray()[np.ix_(fr, fr)]
    ref = np.zeros_like(b)
    ref[fr] = np.linalg.solve(A0, b[fr])
    ev = np.linalg.eigvalsh(A0)
    cond = ev[-1] / ev[0]
    err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
    assert err <= max(1e-13, 100 * cond * U_DF), (err, cond)
    assert not host(x)[lv0.bdof].any()


def test_solve_in_bench_configuration(full):
    """a8-a10 at full size: the benchmark's mixed solve converges to 1e-8; its true
    residual, evaluated cell by cell by the oracle (scalar workloads), meets the same
    bound; the all-FP64 GPU solve needs at most 2 fewer iterations; and the mixed solve
    run on to rtol 1e-11 lies within 1e-7 (relative l2, velocity and pressure) of the
    FP64 solve run to 1e-12 (at rtol 1e-8 both solutions may still be cond * 1e-8 from
    the discrete solution, in any precision)."""
    pb = full.pb
    u, p, info = full.ctx.solve(pb.f, pb.u_bc)
    assert info.converged == 1 and info.res_final <= bench.RTOL * info.res0
    assert not u[np.tile(full.local(full.L - 1).m.boundary_node, full.d)].any()
    if not full.tensor:
        res = stokes_residual(full.local(full.L - 1), pb.f, u, p)
        assert res <= 1.5 * bench.RTOL, res
    opts = dict(full.opts, maxit=300)
    sols = {}
    for key, mode, rtol in (("fp64", A.ALS_MODE_FP64, bench.RTOL), ("fp64_tight", A.ALS_MODE_FP64, 1e-12),
                            ("mixed_tight", A.ALS_MODE_MIXED, 1e-11)):
        ctx = Context(pb.d, pb.n, pb.levels, pb.mu, pb.gamma, mu_eff=full.mu_eff, mode=mode,
                      **dict(opts, rtol=rtol))
        try:
            sols[key] = ctx.solve(pb.f, pb.u_bc)
        finally:
            ctx.close()
        assert sols[key][2].converged == 1, key
    assert info.iterations <= sols["fp64"][2].iterations + 2, (info.iterations, sols["fp64"][2].iterations)
    (um, pm, _), (uf, pf, _) = sols["mixed_tight"], sols["fp64_tight"]
    du = np.linalg.norm(um - uf) / np.linalg.norm(uf)
    dp = np.linalg.norm(pm - pf) / np.linalg.norm(pf)
    assert du <= 1e-7 and dp <= 1e-7, (du, dp)


@pytest.mark.parametrize("workload", ["sinker3d_32", "sinker3d_32_g1e4"])
def test_double_float_setup_equals_fp64_setup(workload):
    """Mixed mode inverts the patches and the coarse operator in double-float arithmetic by
    default; ALS_SETUP_FP64 inverts them in FP64.  On the bench workload (gamma 10, P1) and at
    gamma 1e4 (P2), both solved to rtol 1e-12: the same FGMRES iteration counts (to 1e-8 and
    to 1e-12) and solutions within 1e-9 of each other (measured on a GB300: 8e-13 / 8e-14 at
    gamma 10, 1.1e-11 / 3.9e-13 at gamma 1e4, u / p)."""
    spec = bench.WORKLOADS[workload]
    pb = bench.make_problem(spec)
    mu = [torch.as_tensor(m, device="cuda") for m in pb.mu]
    schur = A.ALS_SCHUR_P2 if spec.get("schur") == "P2" else A.ALS_SCHUR_P1
    res = []
    for setup in (A.ALS_SETUP_AUTO, A.ALS_SETUP_FP64):
        ctx = Context(pb.d, pb.n, pb.levels, mu, pb.gamma, mode=A.ALS_MODE_MIXED, sweeps=spec["sweeps"],
                      schur=schur, setup=setup, rtol=1e-12, maxit=300)
        u, p, info = ctx.solve(pb.f, pb.u_bc)
        h = ctx.solve_history()
        res.append((np.array(u), np.array(p), int(np.flatnonzero(h <= 1e-8 * h[0])[0]), info.iterations))
        ctx.close()
    (u0, p0, a0, b0), (u1, p1, a1, b1) = res
    assert (a0, b0) == (a1, b1)
    assert np.linalg.norm(u0 - u1) <= 1e-9 * np.linalg.norm(u1)
    assert np.linalg.norm(p0 - p1) <= 1e-9 * np.linalg.norm(p1)
