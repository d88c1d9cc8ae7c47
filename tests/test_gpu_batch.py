"""Batches of independent instances (uneven sizes, both dimensions): the batched
solve and the single-launch batched cycle give bitwise the results of the
single-instance calls, which are themselves parity-tested against the oracle."""
import numpy as np
import pytest

from gpu_helpers import context, dev, oracle, rel, sinker

torch = pytest.importorskip("torch")
from paper_2107_00820_gb300 import alstokes as A  # noqa: E402
from oracle.stokes import StokesSolver  # noqa: E402

pytestmark = pytest.mark.gpu

SPECS = [(2, 16, 3, 1e2, 1e4, 31), (2, 32, 4, 1e4, 1e6, 32), (3, 8, 2, 1e2, 1e4, 33), (3, 12, 3, 1e4, 1e6, 34)]


def _instances(mode):
    pbs = [sinker(d, n, L, g, dr, seed) for d, n, L, g, dr, seed in SPECS]
    opts = {"mode": mode, "schur": A.ALS_SCHUR_P2, "rtol": 1e-8}
    ins = [{"dim": pb.d, "n": pb.n, "levels": pb.levels, "coeffs": pb.mu, "gamma": pb.gamma, "options": opts}
           for pb in pbs]
    return pbs, ins, opts


@pytest.mark.parametrize("bmode", [A.ALS_BATCH_MERGED, A.ALS_BATCH_BRANCHES])
@pytest.mark.parametrize("mode", [A.ALS_MODE_FP64, A.ALS_MODE_MIXED])
def test_batch_solve_equals_single_solves(mode, bmode):
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(mode)
    batch = Batch(ins)
    assert batch.mode == A.ALS_BATCH_MERGED   # every instance qualifies
    batch.set_mode(bmode)
    ub, pb_, infos = batch.solve([pb.f for pb in pbs], [pb.u_bc for pb in pbs])
    for i, pb in enumerate(pbs):
        ctx = context(pb, **opts)
        u, p, info = ctx.solve(pb.f, pb.u_bc)
        assert infos[i].converged == 1 and infos[i].iterations == info.iterations
        assert np.array_equal(ub[i], u) and np.array_equal(pb_[i], p)
        ctx.close()
    # the smallest instance against the oracle (FP64: identical iteration counts)
    if mode == A.ALS_MODE_FP64:
        pb = pbs[0]
        s = StokesSolver(oracle(pb, W="Mp_mu"), schur="P2")
        uo, po, its, _ = s.solve(pb.f, pb.u_bc, rtol=1e-8)
        assert infos[0].iterations == its
        assert rel(ub[0], uo) <= 1e-9 and rel(pb_[0], po) <= 1e-8
    batch.close()


@pytest.mark.parametrize("bmode", [A.ALS_BATCH_MERGED, A.ALS_BATCH_BRANCHES])
@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_batch_cycle_equals_single_cycles(prec, bmode):
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(A.ALS_MODE_MIXED)
    batch = Batch(ins)
    batch.set_mode(bmode)
    dt = torch.float64 if prec == A.ALS_PREC_FP64 else torch.float32
    rng = np.random.default_rng(35)
    bs = [dev(rng.standard_normal(s[0]), dt) for s in batch.shapes]
    xs = [torch.zeros_like(b) for b in bs]
    batch.vcycle(bs, xs, prec)
    for i, pb in enumerate(pbs):
        ctx = context(pb, **opts)
        x = torch.zeros_like(bs[i])
        ctx.vcycle(bs[i], x, prec)
        assert torch.equal(x, xs[i]), i
        ctx.close()
    # a second batched launch reuses the graph and gives the same bits
    xs2 = [torch.zeros_like(b) for b in bs]
    batch.vcycle(bs, xs2, prec)
    assert all(torch.equal(a, b) for a, b in zip(xs, xs2))
    batch.close()


def test_merged_cycle_launches_and_tuning():
    """The merged FP32 cycle issues one launch per level operation for each group of
    instances: far fewer kernels than the instances' own cycles together.  The plan's
    tuner timed every distinct grouping and kept the fastest; within each group every
    level's star-kernel variants were timed and the fastest kept."""
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(A.ALS_MODE_MIXED)
    batch = Batch(ins)
    rng = np.random.default_rng(36)
    bs = [dev(rng.standard_normal(s[0]), torch.float32) for s in batch.shapes]
    xs = [torch.zeros_like(b) for b in bs]
    n0 = A.als_kernel_launches()
    batch.vcycle(bs, xs, A.ALS_PREC_FP32)
    merged = A.als_kernel_launches() - n0
    grouping, groups, ms, kern = batch.merged_plan()
    assert kern == merged
    # SPECS: two dimensions, four distinct (dimension, levels) pairs, four shapes; groupings
    # 3 and 4 give the partition of 2 here, so they are not built again
    assert [x > 0 for x in ms] == [True, True, True, False, False]
    assert ms[grouping] == min(x for x in ms if x > 0) and groups == (1, 2, 4)[grouping]
    seen = []
    for g in range(groups):
        members = batch.merged_tune(g, 1)[3]
        seen += members
        lmax = max(pbs[i].levels for i in members)
        for level in range(1, lmax):
            pv, iv, t, _ = batch.merged_tune(g, level)
            assert pv in (0, 1, 2) and iv in (0, 1, 2)
            assert t[pv] == min(t[:3]) and t[3 + iv] == min(t[3:])
        with pytest.raises(A.ALSError):
            batch.merged_tune(g, lmax)
    assert sorted(seen) == list(range(len(pbs)))
    # one launch per operation and level index per group: a group costs the kernels of
    # its deepest instance's own cycle, plus the zeroing launches that replace the
    # single-instance memsets (coarse solve, one interior solve per level)
    single = []
    for i in range(len(pbs)):
        ctx = batch.instance(i)
        x = torch.zeros_like(bs[i])
        ctx.vcycle(bs[i], x, A.ALS_PREC_FP32)
        n0 = A.als_kernel_launches()
        ctx.vcycle(bs[i], x, A.ALS_PREC_FP32)
        single.append(A.als_kernel_launches() - n0)
    bound = 0
    for g in range(groups):
        members = batch.merged_tune(g, 1)[3]
        bound += max(single[i] for i in members) + max(pbs[i].levels for i in members) + 1
    assert merged <= bound, (merged, bound, single)
    if groups < len(pbs):
        assert bound < sum(single), (bound, single)
    batch.close()


@pytest.mark.parametrize("change,why", [({"sweeps": 3}, "sweeps differ from instance 0"),
                                        ({"store": A.ALS_STORE_BF16}, "bfloat16 star storage"),
                                        ({"transfer": A.ALS_TRANSFER_STANDARD}, "transfer differs from instance 0")])
def test_merged_mode_refusal_reasons(change, why):
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(A.ALS_MODE_MIXED)
    ins[1] = dict(ins[1], options=dict(opts, **change))
    batch = Batch(ins)
    assert batch.mode == A.ALS_BATCH_BRANCHES
    with pytest.raises(A.ALSError, match="instance 1 cannot run merged cycles: " + why):
        batch.set_mode(A.ALS_BATCH_MERGED)
    batch.close()


def test_merged_mode_refused_for_an_ineligible_instance():
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(A.ALS_MODE_MIXED)
    ins[2] = dict(ins[2], options=dict(opts, cycle=A.ALS_CYCLE_F))
    batch = Batch(ins)
    assert batch.mode == A.ALS_BATCH_BRANCHES
    with pytest.raises(A.ALSError, match="instance 2 cannot run merged cycles: F-cycle"):
        batch.set_mode(A.ALS_BATCH_MERGED)
    with pytest.raises(A.ALSError, match="unknown batch mode"):
        batch.set_mode(7)
    # the F-cycle instance still cycles (as a graph branch) like its own context
    rng = np.random.default_rng(37)
    bs = [dev(rng.standard_normal(s[0]), torch.float32) for s in batch.shapes]
    xs = [torch.zeros_like(b) for b in bs]
    batch.vcycle(bs, xs, A.ALS_PREC_FP32)
    ctx = context(pbs[2], **dict(opts, cycle=A.ALS_CYCLE_F))
    x = torch.zeros_like(bs[2])
    ctx.vcycle(bs[2], x, A.ALS_PREC_FP32)
    assert torch.equal(x, xs[2])
    ctx.close()
    batch.close()


def test_merged_cycles_beyond_one_launch_table():
    """More instances than one merged launch's parameter table holds (64): every level
    operation splits into several launches, and every instance still gets bitwise its own
    cycle."""
    from paper_2107_00820_gb300 import Batch
    # one (dimension, levels) class
    specs = [(2, 8, 2, 10.0 if i % 2 == 0 else 1e2, 1e2 if i % 3 == 0 else 1e4, 100 + i) for i in range(70)]
    pbs = [sinker(d, n, L, g, dr, seed) for d, n, L, g, dr, seed in specs]
    opts = {"mode": A.ALS_MODE_MIXED, "schur": A.ALS_SCHUR_P2}
    ins = [{"dim": pb.d, "n": pb.n, "levels": pb.levels, "coeffs": pb.mu, "gamma": pb.gamma, "options": opts}
           for pb in pbs]
    batch = Batch(ins)
    assert batch.mode == A.ALS_BATCH_MERGED
    batch.set_grouping(0)                # one group of 70
    with pytest.raises(A.ALSError, match="grouping"):
        batch.set_grouping(5)
    rng = np.random.default_rng(38)
    bs = [dev(rng.standard_normal(s[0]), torch.float32) for s in batch.shapes]
    xs = [torch.zeros_like(b) for b in bs]
    batch.vcycle(bs, xs, A.ALS_PREC_FP32)
    assert batch.merged_plan()[1] == 1
    for i in (0, 1, 63, 64, 68, 69):
        ctx = context(pbs[i], **opts)
        x = torch.zeros_like(bs[i])
        ctx.vcycle(bs[i], x, A.ALS_PREC_FP32)
        assert torch.equal(x, xs[i]), i
        ctx.close()
    batch.close()
