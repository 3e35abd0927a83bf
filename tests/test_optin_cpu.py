"""Per-device bookkeeping of the vote kernel's shared-memory opt-in (host
logic, no GPU): compiled with g++ from csrc/optin.h and run with threads."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_optin_is_tracked_per_device(tmp_path):
    exe = str(tmp_path / "optin_test")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-pthread", "-I",
                           os.path.join(ROOT, "paper_2502_00115_b300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "optin_test.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
