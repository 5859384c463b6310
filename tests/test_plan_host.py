"""Contraction plans on the host (no GPU): builds tests/plan_check.cpp against
libmera.so and runs it.  Dense plans reproduce the contraction's definition;
Z2 charge-sector plans of random symmetric contractions reproduce the dense
ones entry by entry, write exactly the even-charge entries, hold a quarter of
the work and keep the output-layout hints the tensor-core epilogue relies on;
the four real products of the real view of complex operands reproduce complex
contractions (conjugated operands, beta); the library's networks build with
sector plans and real views; the library's leg grading equals the input
generators'."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plans_match_definitions(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    from paper_2007_03638_gb300 import build as b
    lib = b.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "plan_check")
    cmd = [cxx, "-std=c++17", "-O1", os.path.join(ROOT, "tests", "plan_check.cpp"),
           "-I", os.path.join(ROOT, "paper_2007_03638_gb300", "csrc"), "-I", os.path.join(cuda, "include"),
           lib, "-Wl,-rpath," + os.path.dirname(lib), "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.splitlines()
    assert lines[0] == "ok 300"
    assert lines[1] == "complex ok 200"
    assert lines[2] == "networks ok 57"
    # the library grades legs as the input generators do (first half even)
    from paper_2007_03638_gb300 import inputs as inp
    for line in lines[3:]:
        head, vals = line.split(":")
        e = int(head.split()[1])
        assert [int(v) for v in vals.split()] == inp.z2_parities(e).tolist(), line
