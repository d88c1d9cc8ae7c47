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


@pytest.mark.parametrize("mode", [A.ALS_MODE_FP64, A.ALS_MODE_MIXED])
def test_batch_solve_equals_single_solves(mode):
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(mode)
    batch = Batch(ins)
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


@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_batch_cycle_equals_single_cycles(prec):
    from paper_2107_00820_gb300 import Batch
    pbs, ins, opts = _instances(A.ALS_MODE_MIXED)
    batch = Batch(ins)
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
