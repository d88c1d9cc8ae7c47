"""The N > 1 path of bench.py on the CPU with the gloo backend.  The hot path does not
shard (replicas only: every rank solves its own copy of the workload), so the only
multi-process logic is the plumbing: rank discovery from the torchrun environment, the
barrier around the timed region, the maximum of the per-rank step times, the whole-job
value (ranks x DoFs / slowest rank's step time), and the reference arm, which runs on
rank 0 alone while the other ranks exit without work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    bench.Dist._cuda = staticmethod(lambda: False)   # gloo on the host even where a GPU is visible
    d = bench.Dist(world)
    try:
        step_s = 0.10 + 0.05 * rank                # this rank's measured step time
        d.barrier()
        t_step = d.max(step_s)                     # slowest rank sets the job's step time
        dofs = 1000
        value = d.world * dofs / t_step            # whole-job aggregate, as the bench line reports it
        out.put((rank, d.world, d.rank, t_step, value))
    finally:
        d.close()


def test_dist_gloo_two_ranks_max_and_aggregate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, world, drank, t_step, value in res:
        assert world == 2 and drank == rank
        assert t_step == pytest.approx(0.15)          # the max over ranks, on every rank
        assert value == pytest.approx(2 * 1000 / 0.15)
    del torch


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    calls = []
    monkeypatch.setattr(bench, "run_oracle_subprocess", lambda *a, **k: calls.append(a) or [])
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload = "sinker3d_32"
        warmup = 0
        steps = 1
        gpus = 2

    assert bench.reference_arm(Args(), bench._RankOnly()) is None
    assert calls == []                                # rank 1 did no work
