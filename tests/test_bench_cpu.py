"""bench.py's host-side parts, without a GPU: the reference arm's JSON line
(the oracle on the host cores), the clock sampler's parsing (against a fake
nvidia-smi) and the rule that ncu traffic is used only while the recorded
source hash matches the kernel sources."""
import json
import os
import shutil
import stat
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "plain-small", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 3, 3)
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["config"]["workload"] == "plain-q64-2k"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


FAKE_SMI = """#!/bin/sh
echo "GPU-abc, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Active"
echo "GPU-abc, 1950, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
echo "GPU-other, 500, 2070, 100.0, 0x0, Active, Not Active, Not Active, Not Active"
echo "GPU-abc, 2010, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active"
exec sleep 30
"""


def test_clock_sampler_parses_its_gpu_and_cleans_up(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text(FAKE_SMI)
    fake.chmod(fake.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.ClockSampler("GPU-abc")
    c.start()
    for _ in range(100):                    # the fake prints at once, then sleeps
        if os.path.getsize(c.path) > 0 and open(c.path).read().count("\n") >= 4:
            break
        time.sleep(0.05)
    got = c.stop()
    assert got["samples"] == 3                              # the other GPU's line is left out
    assert got["sm_mhz"] == 2010.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)


def test_clock_sampler_without_nvidia_smi(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(None)
    c.start()
    assert c.stop()["reasons"] == ["unsampled"]
    assert not os.path.exists(c.path)


def test_traffic_needs_the_matching_source_hash(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1508_06561_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("hs_device.cuh", "hs_scan.cu", "hs_internal.h"):
        shutil.copy(os.path.join(ROOT, "paper_1508_06561_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles" / "scan_kernel_w.md"
    prof.write_text("source_hash: %s\ntraffic_bytes_per_launch: 123456\n" % h)
    assert bench.recorded_traffic("w") == 123456.0
    prof.write_text("source_hash: %s\ntraffic_bytes_per_launch: 123456\n" % ("0" * 16))
    assert bench.recorded_traffic("w") is None
    assert bench.recorded_traffic("missing") is None
    with open(csrc / "hs_scan.cu", "a") as f:               # any kernel source change voids it
        f.write("\n")
    prof.write_text("source_hash: %s\ntraffic_bytes_per_launch: 123456\n" % h)
    assert bench.recorded_traffic("w") is None
