"""The vote histogram's row and plane stride choice (host logic, no GPU):
compiled with g++ from csrc/strides.h and run."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stride_choice_is_one_to_one_and_spreads_banks(tmp_path):
    exe = str(tmp_path / "strides_test")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_00115_b300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "strides_test.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
