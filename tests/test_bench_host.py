"""Host-side helpers of bench.py, on the CPU: the clock record taken during
the timed steps, and the DRAM traffic read from a committed ncu record that
is tied to the dominant kernel's sources by a digest."""
import os
import sys
import threading

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.proc = _Proc()
    c._t = threading.Thread(target=lambda: None)
    c._t.start()
    c.lines = list(lines)
    return c


NOT = "Not Active"


def test_clock_record_median_max_and_active_reasons():
    lines = [
        "0, 2070, 2070, 910.2, 0x0000000000000000, %s, %s, %s, %s" % (NOT, NOT, NOT, NOT),
        "0, 1965, 2070, 1391.0, 0x0000000000000004, %s, %s, %s, Active" % (NOT, NOT, NOT),
        "0, 2070, 2070, 1002.7, 0x0000000000000000, %s, %s, %s, %s" % (NOT, NOT, NOT, NOT),
        "not a sample",
        "0, [N/A], 2070, 1000, 0x0, %s, %s, %s, %s" % (NOT, NOT, NOT, NOT),
    ]
    r = _sampler(lines).stop()
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_record_names_every_slowdown_seen():
    lines = ["0, 1500, 2070, 700, 0x68, Active, %s, %s, %s" % (NOT, NOT, NOT),
             "0, 1400, 2070, 700, 0x68, %s, Active, Active, %s" % (NOT, NOT)]
    r = _sampler(lines).stop()
    assert r["sm_mhz"] == 1450.0
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def _record(tmp_path, digest, pages=4, dram=1000):
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    (tmp_path / "profiles" / "rec.md").write_text(
        "# a kernel\n\n| kernel | note: with a colon |\n|---|---|\n\n"
        "- pages: %d\n- dram_bytes_per_launch: %d\n- csrc_sha256: %s\n" % (pages, dram, digest))


def test_traffic_record_is_scaled_to_the_pages_while_the_digest_matches(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_digest", lambda: "abc123")
    _record(tmp_path, "abc123", pages=4, dram=1000)
    assert bench.profile_traffic("rec.md", 10) == 2500
    _record(tmp_path, "0ther", pages=4, dram=1000)           # taken from other sources
    assert bench.profile_traffic("rec.md", 10) is None
    assert bench.profile_traffic("missing.md", 10) is None
    (tmp_path / "profiles" / "rec.md").write_text("- pages: 4\n- csrc_sha256: abc123\n")
    assert bench.profile_traffic("rec.md", 10) is None      # no byte count


def test_digest_covers_the_dominant_kernels_sources():
    d = bench.csrc_digest()
    assert len(d) == 64 and int(d, 16) >= 0
    for f in bench.DOMINANT_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_0712_0121_gb300", "csrc", f)), f


def test_reference_arm_prints_one_complete_line():
    """``bench.py --impl reference`` (the oracle on the host cores) prints
    the contract's JSON line on a CPU-only machine."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--cpu-seconds", "0.5"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the other ranks of the reference arm exit 0 without
    work or output."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT="29555")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3", "--cpu-seconds", "0.5"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
