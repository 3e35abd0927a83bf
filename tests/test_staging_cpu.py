"""The rotation pass's shared-memory plan (host logic, no GPU): kernels.cuh
pass_staging and set_chunks, compiled with nvcc into a host program and run.
Every staging layout's chunk stays inside its region for histograms up to the
budget and source counts from 1 to 2^24."""
import os
import subprocess

from paper_2502_00115_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_staging_plan_keeps_every_chunk_in_its_region(tmp_path):
    exe = str(tmp_path / "staging_test")
    subprocess.check_call([build.nvcc(), "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_00115_b300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "staging_test.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
