"""bench.py's host-side contract (no GPU): the clock sampler's parsing of
nvidia-smi samples (a fake nvidia-smi on PATH) and the reference arm, the FP64
oracle timed on the host cores: its JSON line, and the ranks other than 0
exiting without work under torchrun's environment."""
import json
import os
import subprocess
import sys
import time

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fake_smi(tmp_path, rows):
    exe = tmp_path / "nvidia-smi"
    exe.write_text("#!/bin/sh\nprintf '%s'\nexec sleep 30\n" % "".join(r + "\\n" for r in rows))
    exe.chmod(0o755)
    return str(tmp_path)


def test_clock_sampler_reads_median_clock_and_active_reasons(tmp_path, monkeypatch):
    rows = ["0, 1900, 2032, 640.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2032, 2032, 1010.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2000, 2032, 980.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    path = s.path
    c = s.stop()
    assert c == {"sm_mhz": 2000.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(path)


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    path = s.path
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
    assert path is None or not os.path.exists(path)


def _run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=600, cwd=ROOT, env=env)


def test_reference_arm_prints_the_contract_line():
    out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "modelnet_like"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["unit"] == bench.UNIT and d["metric"] == bench.METRIC
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    out = _run_bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                     {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
