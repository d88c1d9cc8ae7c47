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


def test_reference_arm_json_contract():
    """bench.py --impl reference on the host: one JSON line with the base contract's keys,
    the oracle as the reference (kind, cores, sample) and an e2e without host transfers."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "sinker2d_128"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["unit"] == "DoF/s"
    assert rec["higher_is_better"] is True and rec["steps"] == 1 and rec["warmup"] == 0
    assert rec["config"]["workload"] == "sinker2d_128"
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == rec["value"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_clock_sampler_parses_nvidia_smi_samples(tmp_path):
    """The clocks record of the bench line: median SM clock under load, the maximum, and
    every throttle reason seen Active in any sample (sw_power_cap kept, the others flagged)."""
    sys.path.insert(0, ROOT)
    import bench

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    csv = tmp_path / "clocks.csv"
    csv.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                   "0, 2010, 2070, 1350.2, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                   "garbage line\n")
    s = bench.ClockSampler(0)
    s.proc, s.path = Done(), str(csv)
    rec = s.stop()
    assert rec["sm_mhz"] == 2010 and rec["sm_max_mhz"] == 2070 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert not csv.exists()


def test_roofline_inputs(tmp_path, monkeypatch):
    """The roofline fields' inputs: the measured HBM peak from MEASURED_PEAKS.json (else the
    stated 6.8 TB/s fallback), and the committed per-launch DRAM traffic, which is reported
    only while the kernel source still has the hash it was captured on."""
    sys.path.insert(0, ROOT)
    import bench
    peak, kind = bench.measured_peak_hbm()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and 1000 < peak < 20000
    else:
        assert (peak, kind) == (6800.0, "fallback")
    assert bench.stored_traffic("k_patch_apply_f32_fine", "sinker3d_32") > 0
    assert bench.stored_traffic("k_patch_apply_f32_fine", "no_such_workload") is None
    # a source that no longer matches its recorded hash gives no traffic
    fake = tmp_path / "profiles"
    fake.mkdir()
    (tmp_path / "src.cu").write_text("changed")
    (fake / "traffic.txt").write_text("k w src.cu 0000000000000000 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.stored_traffic("k", "w") is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.measured_peak_hbm() == (6800.0, "fallback")
