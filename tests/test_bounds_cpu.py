"""The bound behind the vote's 16-bit counters (host logic, no GPU): csrc/bounds.h
compiled with g++ and checked against a brute-force count of the points in
every cube of side delta on random, clustered and cell-edge point sets."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counter_bound_covers_every_cube(tmp_path):
    exe = str(tmp_path / "bounds_test")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_00115_b300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "bounds_test.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
