"""Host logic of bench.py, on the CPU: the reference arm's JSON line, the clock record
taken during the timed region, and the inputs of the roofline fields."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    live = bench.stored_traffic("k_patch_apply_f32_fine", "sinker3d_32")
    assert live is None or live > 0          # None once the kernel source has changed
    assert bench.stored_traffic("k_patch_apply_f32_fine", "no_such_workload") is None
    # a source that matches its recorded hash gives the traffic; a changed one gives none
    import hashlib
    fake = tmp_path / "profiles"
    fake.mkdir()
    (tmp_path / "src.cu").write_text("kernel")
    sha = hashlib.sha256(b"kernel").hexdigest()[:16]
    (fake / "traffic.txt").write_text(f"k w src.cu {sha} 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.stored_traffic("k", "w") == 123.0
    (tmp_path / "src.cu").write_text("changed")
    assert bench.stored_traffic("k", "w") is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "nowhere"))
    assert bench.measured_peak_hbm() == (6800.0, "fallback")
